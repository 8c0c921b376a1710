// fft_core.cuh -- register/shared-memory FFT on pencils (sm_103a).
//
// Every length L = 2^p (8 <= L <= 1024) is split once, L = R1 * R2 with
// R1 = 2^floor(p/2) and R2 = L / R1 (R2 = R1 or 2 R1), and transformed in two
// radix stages with ONE shared-memory exchange between them (the four-step /
// Stockham split of Cooley-Tukey):
//
//   stage 1: R2 DFTs of size R1 over x[n2 + R2 n1]            (registers)
//   exchange through shared memory                           (one barrier)
//   twiddle  exp(DIR 2 pi i k1 n2 / L)                        (table)
//   stage 2: R1 DFTs of size R2 over the twiddled values      (registers)
//
// A pencil is worked by NT = R1 threads holding V = R2 complex values each:
// thread j holds v[u] = x[j + u*NT] before the transform and X[j + u*NT]
// after it (natural order in and out), so callers fuse elementwise work
// (clips, masks, reductions) on the registers.  The register DFTs of size
// 2..32 are split recursively into sizes 4 and 8 with their internal twiddles
// as compile-time constants.
//
// A "tile" is W pencils interleaved in shared memory (element l of pencil w
// at row l, column w; a row is W complex values) with one padding row after
// every R1 rows: the stage-1 stores (rows R1-strided across threads) and the
// stage-2 loads (consecutive rows across threads) both stay within the
// minimum number of shared-memory wavefronts.  One buffer per tile; the
// barrier before an exchange that reuses it is taken only when needed.  A
// tile of at most 32 threads lies inside one warp and synchronises with
// __syncwarp instead of a block barrier.
//
// The transform is the unnormalised DFT of Eq. 1, X_k = sum_n x_n w^{nk},
// w = exp(DIR 2 pi i / L), DIR = -1 forward, +1 inverse (no 1/L).
//
// Twiddle table of length L: exp(-2 pi i k1 t / L) for k1 < R1, t = 1..R2-1
// at entry tw_index(k1, t) = ((t-1)/2) 2 R1 + 2 k1 + (t-1)%2: factors t and
// t+1 of one k1 are adjacent (one 128-bit load in float32) and, for a fixed
// pair, the k1 of consecutive threads are consecutive, so a warp's loads hit
// distinct banks.  Computed on the host in long double and rounded once; the
// inverse uses the conjugates.
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
// float32 complex add/sub as one packed two-lane operation (the f32x2 ops
// of sm_100 and later: one instruction for both components, the same
// round-to-nearest results as two scalar operations; a - b is computed as
// b * (-1) + a, exact up to the single rounding of the sum).  Products that
// mix the two components of a value (twiddles, multiplication by i) stay
// scalar: the lane swaps they would need cost more than they save.
template <>
__device__ __forceinline__ float2 add<float>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <>
__device__ __forceinline__ float2 sub<float>(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
// a + DIR i t and a - DIR i t (the odd outputs of a radix-4 butterfly)
template <typename T, int DIR>
__device__ __forceinline__ v2<T> add_mul_i(v2<T> a, v2<T> t) {
  if constexpr (DIR < 0) return mk<T>(a.x + t.y, a.y - t.x);
  else return mk<T>(a.x - t.y, a.y + t.x);
}
template <typename T, int DIR>
__device__ __forceinline__ v2<T> sub_mul_i(v2<T> a, v2<T> t) {
  if constexpr (DIR < 0) return mk<T>(a.x - t.y, a.y + t.x);
  else return mk<T>(a.x + t.y, a.y - t.x);
}
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

// cos(2 pi r / 32) for r = 0..8 (decimal values of the exact constants).
__host__ __device__ constexpr double cos32_oct(int r) {
  return r == 0 ? 1.0 : r == 1 ? 0.98078528040323044913 : r == 2 ? 0.92387953251128675613
       : r == 3 ? 0.83146961230254523708 : r == 4 ? 0.70710678118654752440
       : r == 5 ? 0.55557023301960222474 : r == 6 ? 0.38268343236508977173
       : r == 7 ? 0.19509032201612826785 : 0.0;
}
// cos and sin of 2 pi m / 32 for any integer m, by quadrant.
__host__ __device__ constexpr double cos32(int m) {
  return ((m & 31) >> 3) == 0 ? cos32_oct(m & 7) : ((m & 31) >> 3) == 1 ? -cos32_oct(8 - (m & 7))
       : ((m & 31) >> 3) == 2 ? -cos32_oct(m & 7) : cos32_oct(8 - (m & 7));
}
__host__ __device__ constexpr double sin32(int m) { return cos32(m - 8); }

// a * exp(DIR 2 pi i m / 32); m is a constant after unrolling, so every
// branch but one folds away.  Multiples of pi/4 take the cheap forms.
template <typename T, int DIR>
__device__ __forceinline__ v2<T> mul_w32(v2<T> a, int m) {
  m &= 31;
  if (m == 0) return a;
  if (m == 8) return mul_i<T, DIR>(a);
  if (m == 16) return mk<T>(-a.x, -a.y);
  if (m == 24) return mul_i<T, -DIR>(a);
  if (m == 4) return mul_w8_1<T, DIR>(a);
  if (m == 12) return mul_w8_3<T, DIR>(a);
  if (m == 20) { const v2<T> b = mul_w8_1<T, DIR>(a); return mk<T>(-b.x, -b.y); }
  if (m == 28) { const v2<T> b = mul_w8_3<T, DIR>(a); return mk<T>(-b.x, -b.y); }
  const T c = (T)cos32(m), s = (T)(DIR * sin32(m));
  return mk<T>(a.x * c - a.y * s, a.y * c + a.x * s);
}

// In-register DFTs in natural output order.
template <typename T, int DIR>
__device__ __forceinline__ void dft4(v2<T>& a0, v2<T>& a1, v2<T>& a2, v2<T>& a3) {
  v2<T> s02 = add<T>(a0, a2), d02 = sub<T>(a0, a2);
  v2<T> s13 = add<T>(a1, a3), t13 = sub<T>(a1, a3);
  a0 = add<T>(s02, s13); a2 = sub<T>(s02, s13);
  a1 = add_mul_i<T, DIR>(d02, t13); a3 = sub_mul_i<T, DIR>(d02, t13);
}
template <typename T, int DIR>
__device__ __forceinline__ void dft8(v2<T> (&a)[8]) {
  // even/odd split: E = DFT4(a0,a2,a4,a6), O = DFT4(a1,a3,a5,a7)
  dft4<T, DIR>(a[0], a[2], a[4], a[6]);
  dft4<T, DIR>(a[1], a[3], a[5], a[7]);
  v2<T> o1 = mul_w8_1<T, DIR>(a[3]);
  v2<T> o3 = mul_w8_3<T, DIR>(a[7]);
  v2<T> e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6], o0 = a[1], t2 = a[5];
  a[0] = add<T>(e0, o0); a[4] = sub<T>(e0, o0);
  a[1] = add<T>(e1, o1); a[5] = sub<T>(e1, o1);
  a[2] = add_mul_i<T, DIR>(e2, t2); a[6] = sub_mul_i<T, DIR>(e2, t2);
  a[3] = add<T>(e3, o3); a[7] = sub<T>(e3, o3);
}

template <int R, typename T, int DIR>
__device__ __forceinline__ void dftN(v2<T> (&x)[R]);

// DFT of size N = A * B: B DFTs of size A over x[b + B a], internal twiddles
// w_N^{b k1}, A DFTs of size B, output k = k1 + A k2 (Cooley-Tukey).
template <typename T, int DIR, int A, int B>
__device__ __forceinline__ void dft_ab(v2<T> (&x)[A * B]) {
  constexpr int N = A * B;
  static_assert(N <= 32, "internal twiddles are tabulated in 32nds");
#pragma unroll
  for (int b = 0; b < B; ++b) {
    v2<T> t[A];
#pragma unroll
    for (int a = 0; a < A; ++a) t[a] = x[b + B * a];
    dftN<A, T, DIR>(t);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) x[b + B * k1] = mul_w32<T, DIR>(t[k1], b * k1 * (32 / N));
  }
  v2<T> o[N];
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) {
    v2<T> t[B];
#pragma unroll
    for (int b = 0; b < B; ++b) t[b] = x[b + B * k1];
    dftN<B, T, DIR>(t);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) o[k1 + A * k2] = t[k2];
  }
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = o[i];
}

template <int R, typename T, int DIR>
__device__ __forceinline__ void dftN(v2<T> (&x)[R]) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    const v2<T> a = x[0];
    x[0] = add<T>(a, x[1]);
    x[1] = sub<T>(a, x[1]);
  } else if constexpr (R == 4) {
    dft4<T, DIR>(x[0], x[1], x[2], x[3]);
  } else if constexpr (R == 8) {
    dft8<T, DIR>(x);
  } else if constexpr (R == 16) {
    dft_ab<T, DIR, 4, 4>(x);
  } else {
    static_assert(R == 32, "register DFT sizes 1..32");
    dft_ab<T, DIR, 8, 4>(x);
  }
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

// The two-stage split of length L.
template <int L>
struct F2 {
  static_assert(L >= 8 && L <= 1024 && (L & (L - 1)) == 0, "L must be a power of two in [8, 1024]");
  static constexpr int lg = ilog2(L);
  static constexpr int lg1 = lg / 2;
  static constexpr int R1 = 1 << lg1;     // stage-1 size = threads per pencil
  static constexpr int R2 = L / R1;       // stage-2 size = values per thread
  static constexpr int NT = R1, V = R2;
  static constexpr int NB1 = R2 / R1;     // stage-1 DFTs per thread (1 or 2)
  static constexpr int ROWS = L + R2;     // rows of one tile buffer (padding included)
  // buffer row of natural element l
  __host__ __device__ static constexpr int row(int l) { return l + (l >> lg1); }
};
// Host-side values of the same split.
inline int f2_nt(int L) { return 1 << (ilog2(L) / 2); }
inline int f2_v(int L) { return L / f2_nt(L); }
// Table entry of factor t (1 <= t < R2) of stage-2 row k1 (layout above).
__host__ __device__ constexpr int tw_index(int R1, int k1, int t) {
  return ((t - 1) >> 1) * 2 * R1 + 2 * k1 + ((t - 1) & 1);
}

// Pencils per tile of the strided passes: 64-byte rows (8 float32 or 4
// float64 complex values).
template <typename T> struct TileW { static constexpr int value = 16 / (int)sizeof(T) * 2; };

// A thread's view of its pencil's column in the tile buffer.
template <typename T, int L, int W_>
struct Tile {
  static constexpr int W = W_;
  static constexpr int TPT = F2<L>::NT * W;       // threads of the tile
  static constexpr int ELEMS = F2<L>::ROWS * W;   // complex values of the buffer
  v2<T>* p;    // buffer + w
  bool used;   // an earlier exchange has read the buffer
  __device__ __forceinline__ static void sync() {
    if constexpr (TPT <= 32) __syncwarp();
    else __syncthreads();
  }
  // before storing: wait until every thread has read the previous exchange
  __device__ __forceinline__ void begin() {
    if (used) sync();
  }
  __device__ __forceinline__ void done() { used = true; }
  __device__ __forceinline__ v2<T>* buf() const { return p; }
  // natural element l of this pencil / of the pencil `dw` columns away
  __device__ __forceinline__ v2<T>& at(int l) const { return p[F2<L>::row(l) * W]; }
  __device__ __forceinline__ v2<T>& at_other(int l, int dw) const { return p[F2<L>::row(l) * W + dw]; }
};

// Full length-L transform of the thread's pencil (all threads of the tile
// must call it).  tw: the length-L twiddle table (shared memory).
template <typename T, int L, int DIR, class TL>
__device__ __forceinline__ void fft_pencil(v2<T> (&v)[F2<L>::V], int j, const v2<T>* __restrict__ tw,
                                           TL& tl) {
  using F = F2<L>;
  constexpr int R1 = F::R1, R2 = F::R2, NB1 = F::NB1, W = TL::W;
  tl.begin();
  v2<T>* buf = tl.buf();
#pragma unroll
  for (int b = 0; b < NB1; ++b) {
    v2<T> x[R1];
#pragma unroll
    for (int t = 0; t < R1; ++t) x[t] = v[b + t * NB1];
    dftN<R1, T, DIR>(x);
    // output t of stage-1 DFT n2 = j + b R1 is element n2 R1 + t
    const int r0 = (j + b * R1) * (R1 + 1);
#pragma unroll
    for (int t = 0; t < R1; ++t) buf[(r0 + t) * W] = x[t];
  }
  TL::sync();
  // element j + t R1 (row j + t (R1 + 1)), twiddled by w_L^{j t}
#pragma unroll
  for (int t = 0; t < R2; ++t) v[t] = buf[(j + t * (R1 + 1)) * W];
  tl.done();
  if constexpr (sizeof(T) == 4) {
    const float4* q = reinterpret_cast<const float4*>(tw) + j;
#pragma unroll
    for (int i = 0; i < R2 / 2; ++i) {
      const float4 f = q[i * R1];   // factors 2i+1, 2i+2 of row j
      v[2 * i + 1] = twmul<T, DIR>(v[2 * i + 1], mk<T>(f.x, f.y));
      if (2 * i + 2 < R2) v[2 * i + 2] = twmul<T, DIR>(v[2 * i + 2], mk<T>(f.z, f.w));
    }
  } else {
#pragma unroll
    for (int t = 1; t < R2; ++t) v[t] = twmul<T, DIR>(v[t], tw[tw_index(R1, j, t)]);
  }
  dftN<R2, T, DIR>(v);
}

// Exchange in natural order: every thread stores its registers, the tile
// synchronises, and the caller reads other elements with at()/at_other();
// the caller then calls tl.done().  Used where an elementwise step needs
// X[-k] next to X[k].
template <typename T, int L, class TL>
__device__ __forceinline__ void store_nat(const v2<T> (&v)[F2<L>::V], int j, TL& tl) {
  constexpr int R1 = F2<L>::R1, W = TL::W;
  tl.begin();
  v2<T>* dst = tl.buf();
#pragma unroll
  for (int u = 0; u < F2<L>::V; ++u) dst[(j + u * (R1 + 1)) * W] = v[u];
  TL::sync();
}

}  // namespace ffcz
