// fft_core.cuh -- register/shared-memory Stockham FFT on pencils (sm_103a).
//
// One "tile" is W pencils of length L (a power of two, 8..1024) processed by
// (L/8)*W threads (W: see TileW).  Thread (j, w) with w = tid % W, j = tid / W holds eight
// complex values of pencil w in registers: v[u] = x[j + u*L/8] (u = 0..7).
// Between the radix stages the values go through shared memory, pencils
// interleaved (element l of pencil w at row l, column w; rows of W elements
// are 64 bytes) with one padding row after every 8 rows.  The padding keeps
// every stage permutation within ~6% of the minimum number of shared-memory
// wavefronts, and, unlike an XOR swizzle, gives each thread addresses of the
// form base + compile-time offset.  Two tile buffers alternate ("ping-pong"),
// so one barrier per exchange suffices.
//
// The transform is the unnormalised DFT of Eq. 1, X_k = sum_n x_n w^{nk},
// w = exp(DIR 2 pi i / L), DIR = -1 forward, +1 inverse (no 1/L), in the
// Stockham autosort formulation (Cooley-Tukey with a permuting store after
// every stage, natural order in and out).  Radix schedule: all radix-8 when
// 3 | log2 L; otherwise one (log2 L = 3a+2) or two (3a+1) radix-4 stages
// first.  After the last stage thread j again holds X[j + u*L/8], so callers
// can fuse elementwise work (clips, masks, reductions) on the registers.
//
// Twiddles: per stage (R, NS), for k < NS the factors exp(-2 pi i k t/(R NS)),
// t = 1..R-1, stored contiguously (padded to 8 or 4 entries) so a thread
// fetches its stage's factors with 128-bit loads.  They are computed on the
// host in long double and rounded once; the inverse uses the conjugates.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ffcz {

template <typename T> struct V2T;
template <> struct V2T<float> { using type = float2; };
template <> struct V2T<double> { using type = double2; };
template <typename T> using v2 = typename V2T<T>::type;

template <typename T>
__device__ __forceinline__ v2<T> mk(T x, T y) { v2<T> r; r.x = x; r.y = y; return r; }
template <typename T>
__device__ __forceinline__ v2<T> add(v2<T> a, v2<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ v2<T> sub(v2<T> a, v2<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ v2<T> cmul(v2<T> a, v2<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ v2<T> cmulc(v2<T> a, v2<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T, int DIR>
__device__ __forceinline__ v2<T> twmul(v2<T> a, v2<T> w) {
  if constexpr (DIR < 0) return cmul<T>(a, w);
  else return cmulc<T>(a, w);
}

template <typename T> __device__ __forceinline__ T rsqrt2();
template <> __device__ __forceinline__ float rsqrt2<float>() { return 0.70710678118654752440f; }
template <> __device__ __forceinline__ double rsqrt2<double>() { return 0.70710678118654752440; }

// Multiply by DIR*i (-i forward, +i inverse).
template <typename T, int DIR>
__device__ __forceinline__ v2<T> mul_i(v2<T> a) {
  if constexpr (DIR < 0) return mk<T>(a.y, -a.x);
  else return mk<T>(-a.y, a.x);
}
// Multiply by exp(DIR i pi/4) and exp(DIR 3 i pi/4).
template <typename T, int DIR>
__device__ __forceinline__ v2<T> mul_w8_1(v2<T> a) {
  const T s = rsqrt2<T>();
  if constexpr (DIR < 0) return mk<T>((a.x + a.y) * s, (a.y - a.x) * s);
  else return mk<T>((a.x - a.y) * s, (a.x + a.y) * s);
}
template <typename T, int DIR>
__device__ __forceinline__ v2<T> mul_w8_3(v2<T> a) {
  const T s = rsqrt2<T>();
  if constexpr (DIR < 0) return mk<T>((a.y - a.x) * s, -(a.x + a.y) * s);
  else return mk<T>(-(a.x + a.y) * s, (a.x - a.y) * s);
}

// In-register DFTs of size 4 and 8 in natural output order.
template <typename T, int DIR>
__device__ __forceinline__ void dft4(v2<T>& a0, v2<T>& a1, v2<T>& a2, v2<T>& a3) {
  v2<T> s02 = add<T>(a0, a2), d02 = sub<T>(a0, a2);
  v2<T> s13 = add<T>(a1, a3), d13 = mul_i<T, DIR>(sub<T>(a1, a3));
  a0 = add<T>(s02, s13); a2 = sub<T>(s02, s13);
  a1 = add<T>(d02, d13); a3 = sub<T>(d02, d13);
}
template <typename T, int DIR>
__device__ __forceinline__ void dft8(v2<T> (&a)[8]) {
  // even/odd split: E = DFT4(a0,a2,a4,a6), O = DFT4(a1,a3,a5,a7)
  dft4<T, DIR>(a[0], a[2], a[4], a[6]);
  dft4<T, DIR>(a[1], a[3], a[5], a[7]);
  v2<T> o1 = mul_w8_1<T, DIR>(a[3]);
  v2<T> o2 = mul_i<T, DIR>(a[5]);
  v2<T> o3 = mul_w8_3<T, DIR>(a[7]);
  v2<T> e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6], o0 = a[1];
  a[0] = add<T>(e0, o0); a[4] = sub<T>(e0, o0);
  a[1] = add<T>(e1, o1); a[5] = sub<T>(e1, o1);
  a[2] = add<T>(e2, o2); a[6] = sub<T>(e2, o2);
  a[3] = add<T>(e3, o3); a[7] = sub<T>(e3, o3);
}
template <int R, typename T, int DIR>
__device__ __forceinline__ void dftR(v2<T> (&x)[R]) {
  if constexpr (R == 4) dft4<T, DIR>(x[0], x[1], x[2], x[3]);
  else dft8<T, DIR>(x);
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

// Pencils per tile: float64 tiles use 4 (64-byte rows); float32 tiles use
// FFCZ_W32 pencils (4: 32-byte rows, CTAs half the size and twice as many
// resident; 8: 64-byte rows).
#ifndef FFCZ_W32
#define FFCZ_W32 8
#endif
template <typename T> struct TileW { static constexpr int value = 4; };
template <> struct TileW<float> { static constexpr int value = FFCZ_W32; };

// Radix schedule and twiddle-table layout for length L (host and device).
template <int L>
struct Sched {
  static constexpr int lg = ilog2(L), a = lg / 3, b = lg % 3;
  static constexpr int nst = (b == 0) ? a : a + 1;
  __host__ __device__ static constexpr int radix(int s) {
    return b == 0 ? 8 : (b == 2 ? (s == 0 ? 4 : 8) : (s < 2 ? 4 : 8));
  }
  __host__ __device__ static constexpr int ns(int s) {
    int n = 1;
    for (int i = 0; i < s; ++i) n *= radix(i);
    return n;
  }
  __host__ __device__ static constexpr int sp(int s) { return radix(s) == 8 ? 8 : 4; }
  __host__ __device__ static constexpr int twoff(int s) {
    int o = 0;
    for (int i = 1; i < s; ++i) o += ns(i) * sp(i);
    return o;
  }
  static constexpr int twsize = twoff(nst) > 0 ? twoff(nst) : 4;
};

// Row index with one padding row after every 8 rows.
__host__ __device__ constexpr int pidx(int l) { return l + (l >> 3); }

// A thread's view of its pencil in two ping-pong tile buffers.
template <typename T, int L, int W_ = TileW<T>::value>
struct Tile {
  static constexpr int W = W_;
  static constexpr int ROWS = L + L / 8;
  static constexpr int ELEMS = ROWS * W;   // one buffer
  v2<T>* p0;  // buffer used by even exchanges (+ w)
  v2<T>* p1;  // buffer used by odd exchanges (+ w)
  int ph;     // buffer the next exchange uses
  __device__ __forceinline__ v2<T>* buf() const { return ph ? p1 : p0; }
  __device__ __forceinline__ void flip() { ph ^= 1; }
  // element l of this pencil / of the pencil `dw` columns away, current buffer
  __device__ __forceinline__ v2<T>& at(int l) const { return buf()[pidx(l) * W]; }
  __device__ __forceinline__ v2<T>& at_other(int l, int dw) const { return buf()[pidx(l) * W + dw]; }
};

// Natural-order row index of register u of thread j: pidx(j + u*NT).
template <int NT>
__device__ __forceinline__ int nat(int jb, int j, int u) {
  if constexpr (NT % 8 == 0) return jb + u * (NT + NT / 8);
  else return pidx(j + u * NT);
}

// One Stockham stage S of the schedule: radix R, sub-transform size NS.
// Thread j owns 8/R butterflies j' = j + b*L/8; butterfly j' takes
// x[j' + t*L/R] (registers v[b + t*8/R]); after the twiddles
// exp(DIR 2 pi i k t/(R NS)), k = j' mod NS, and the R-point DFT, output t
// goes to row (j'/NS)*R*NS + k + t*NS.  The last stage keeps the outputs in
// registers: they are then x[j + u*L/8] again.
template <typename T, int L, int DIR, int S, class TL>
__device__ __forceinline__ void stockham_stage(v2<T> (&v)[8], int j, int jb,
                                               const v2<T>* __restrict__ tw, TL& tl) {
  using SC = Sched<L>;
  constexpr int R = SC::radix(S), NS = SC::ns(S), NT = L / 8, NB = 8 / R, W = TL::W;
  constexpr bool last = (S == SC::nst - 1);
  v2<T>* dst = tl.buf();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int jp = j + b * NT;
    const int k = jp & (NS - 1);
    v2<T> x[R];
#pragma unroll
    for (int t = 0; t < R; ++t) x[t] = v[b + t * NB];
    if constexpr (NS > 1) {
      // factors t = 1..R-1 of this butterfly, fetched two at a time
      const v2<T>* twk = tw + SC::twoff(S) + k * SC::sp(S);
      if constexpr (sizeof(T) == 4) {
        const float4* q = reinterpret_cast<const float4*>(twk);
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
          const float4 f = q[i];
          if (2 * i + 1 < R) x[2 * i + 1] = twmul<T, DIR>(x[2 * i + 1], mk<T>(f.x, f.y));
          if (2 * i + 2 < R) x[2 * i + 2] = twmul<T, DIR>(x[2 * i + 2], mk<T>(f.z, f.w));
        }
      } else {
#pragma unroll
        for (int t = 1; t < R; ++t) x[t] = twmul<T, DIR>(x[t], twk[t - 1]);
      }
    }
    dftR<R, T, DIR>(x);
    if constexpr (last) {
#pragma unroll
      for (int t = 0; t < R; ++t) v[b + t * NB] = x[t];
    } else {
      const int o = (jp / NS) * (R * NS) + k;
      if constexpr (NS >= 8) {
        const int base = o + (o >> 3);
#pragma unroll
        for (int t = 0; t < R; ++t) dst[(base + t * (NS + NS / 8)) * W] = x[t];
      } else if constexpr (NS == 4) {
        const int base = o + (jp >> 2) * (R / 2);
#pragma unroll
        for (int t = 0; t < R; ++t) dst[(base + 4 * t + (t >> 1)) * W] = x[t];
      } else {
        const int base = jp * R + (R == 8 ? jp : (jp >> 1));
#pragma unroll
        for (int t = 0; t < R; ++t) dst[(base + t) * W] = x[t];
      }
    }
  }
  if constexpr (!last) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = dst[nat<NT>(jb, j, u) * W];
    tl.flip();
  }
}

template <typename T, int L, int DIR, int S, class TL>
__device__ __forceinline__ void stages_from(v2<T> (&v)[8], int j, int jb, const v2<T>* __restrict__ tw,
                                            TL& tl) {
  if constexpr (S < Sched<L>::nst) {
    stockham_stage<T, L, DIR, S, TL>(v, j, jb, tw, tl);
    stages_from<T, L, DIR, S + 1, TL>(v, j, jb, tw, tl);
  }
}

// Full length-L transform of the thread's pencil.  Every thread of the CTA
// must call it (it synchronises the block between stages).  `jb` is
// pidx(j) (precomputed by the caller).
template <typename T, int L, int DIR, class TL>
__device__ __forceinline__ void fft_pencil(v2<T> (&v)[8], int j, int jb, const v2<T>* __restrict__ tw,
                                           TL& tl) {
  static_assert(L >= 8 && (L & (L - 1)) == 0, "L must be a power of two >= 8");
  stages_from<T, L, DIR, 0, TL>(v, j, jb, tw, tl);
}

// Exchange: every thread stores its natural-order registers, the block
// synchronises, and `f(l)` below reads other rows; afterwards the buffers
// flip.  Used where an elementwise step needs X[-k] next to X[k].
template <typename T, int L, class TL>
__device__ __forceinline__ void store_nat(const v2<T> (&v)[8], int j, int jb, TL& tl) {
  constexpr int NT = L / 8, W = TL::W;
  v2<T>* dst = tl.buf();
#pragma unroll
  for (int u = 0; u < 8; ++u) dst[nat<NT>(jb, j, u) * W] = v[u];
  __syncthreads();
}

}  // namespace ffcz
