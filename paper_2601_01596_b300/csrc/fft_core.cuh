// fft_core.cuh -- register/shared-memory Stockham FFT on pencils (sm_103a).
//
// One "tile" is W pencils of length L (a power of two, 8..1024) processed by
// (L/8)*W threads.  Thread (j, w) with w = tid % W, j = tid / W holds eight
// complex values of pencil w in registers: v[u] = x[j + u*L/8] (u = 0..7).
// Between the radix stages the values go through shared memory; the pencils
// are interleaved there so that a half-warp touching the same index of its
// W pencils reads one 64-byte row.  Two rows share a 128-byte line and a
// one-bit XOR swizzle on the line half keeps the stage permutations nearly
// free of bank conflicts (about 5% extra wavefronts, all L).
//
// The transform is the unnormalised DFT of Eq. 1, X_k = sum_n x_n w^{nk},
// w = exp(DIR 2 pi i / L), DIR = -1 forward, +1 inverse (no 1/L).  It is the
// Stockham autosort formulation (Cooley-Tukey with a permuting store at
// every stage, so input and output are in natural order): a first radix-2 or
// radix-4 stage when log2(L) is not a multiple of 3, then radix-8 stages.
// After the last stage thread j again holds X[j + u*L/8], which lets callers
// fuse elementwise work (clips, masks, reductions) on the registers.
//
// Twiddles come from a table of exp(-2 pi i m / L), m < L, computed on the
// host in long double and rounded once; the inverse uses the conjugate.
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

// In-register DFTs of size 2, 4, 8 in natural output order.
template <typename T, int DIR>
__device__ __forceinline__ void dft2(v2<T>& a0, v2<T>& a1) {
  v2<T> t = a0; a0 = add<T>(t, a1); a1 = sub<T>(t, a1);
}
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
  if constexpr (R == 2) dft2<T, DIR>(x[0], x[1]);
  else if constexpr (R == 4) dft4<T, DIR>(x[0], x[1], x[2], x[3]);
  else dft8<T, DIR>(x);
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

// Shared-memory view of one pencil of an interleaved tile.
// Rows of W elements are 64 bytes; element (l, w) of the tile lives at
// line (l >> 1), half ((l & 1) ^ swz(l >> 1)), column w.
template <typename T>
struct Slot {
  static constexpr int W = 64 / (int)sizeof(v2<T>);
  v2<T>* base;  // tile base
  int w;        // pencil index in the tile
  __device__ __forceinline__ int idx(int l) const {
    int m = l >> 1;
    int half = (l & 1) ^ ((m ^ (m >> 2)) & 1);
    return m * (2 * W) + half * W + w;
  }
  __device__ __forceinline__ v2<T>& at(int l) const { return base[idx(l)]; }
};

// One Stockham stage: radix R, sub-transform size NS (R*NS divides L).
// Every thread owns 8/R butterflies: j' = j + b*L/8, b < 8/R; butterfly j'
// takes x[j' + t*L/R] (registers v[b + t*8/R]) and, after the twiddle
// exp(DIR 2 pi i k t / (R NS)), k = j' mod NS, and the R-point DFT, puts
// output t at position (j'/NS)*R*NS + k + t*NS.  The last stage keeps the
// outputs in registers: they are then x[j + u*L/8] again.
template <typename T, int L, int DIR, int R, int NS>
__device__ __forceinline__ void stockham_stage(v2<T> (&v)[8], int j, const v2<T>* __restrict__ tw,
                                               const Slot<T>& sm) {
  constexpr int NT = L / 8, NB = 8 / R;
  constexpr bool last = (R * NS == L);
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int jp = j + b * NT;
    const int k = jp & (NS - 1);
    v2<T> x[R];
#pragma unroll
    for (int t = 0; t < R; ++t) x[t] = v[b + t * NB];
    if constexpr (NS > 1) {
#pragma unroll
      for (int t = 1; t < R; ++t) {
        const int m = k * t * (L / (R * NS));
        x[t] = twmul<T, DIR>(x[t], tw[m]);
      }
    }
    dftR<R, T, DIR>(x);
    if constexpr (last) {
#pragma unroll
      for (int t = 0; t < R; ++t) v[b + t * NB] = x[t];
    } else {
      const int o = (jp / NS) * (R * NS) + k;
#pragma unroll
      for (int t = 0; t < R; ++t) sm.at(o + t * NS) = x[t];
    }
  }
  if constexpr (!last) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = sm.at(j + u * NT);
    __syncthreads();
  }
}

template <typename T, int L, int DIR, int NS>
__device__ __forceinline__ void radix8_stages(v2<T> (&v)[8], int j, const v2<T>* __restrict__ tw,
                                              const Slot<T>& sm) {
  if constexpr (NS < L) {
    stockham_stage<T, L, DIR, 8, NS>(v, j, tw, sm);
    radix8_stages<T, L, DIR, NS * 8>(v, j, tw, sm);
  }
}

// Full length-L transform of the thread's pencil.  Must be called by every
// thread of the CTA (it synchronises the block between stages).
template <typename T, int L, int DIR>
__device__ __forceinline__ void fft_pencil(v2<T> (&v)[8], int j, const v2<T>* __restrict__ tw,
                                           const Slot<T>& sm) {
  static_assert(L >= 8 && (L & (L - 1)) == 0, "L must be a power of two >= 8");
  constexpr int b = ilog2(L) % 3;
  if constexpr (b == 0) {
    radix8_stages<T, L, DIR, 1>(v, j, tw, sm);
  } else {
    stockham_stage<T, L, DIR, (1 << b), 1>(v, j, tw, sm);
    radix8_stages<T, L, DIR, (1 << b)>(v, j, tw, sm);
  }
}

}  // namespace ffcz
