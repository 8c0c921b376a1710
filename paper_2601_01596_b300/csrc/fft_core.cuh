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
// inverse uses the conjugates.  The FP64 table holds the factors t >= R2/2 in
// the tangent form (c, s/c) that the fused first butterfly layer of stage 2
// reads (fold_rt; host side: f64_stage_entry).
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

template <int R, int DIR>
__device__ __forceinline__ void dftN_f64(double2 (&x)[R]);

template <int R, typename T, int DIR>
__device__ __forceinline__ void dftN(v2<T> (&x)[R]) {
  if constexpr (sizeof(T) == 8) {
    dftN_f64<R, DIR>(x);
  } else if constexpr (R == 1) {
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

// ---------------------------------------------------------------------------
// FP64 register DFTs with the twiddle products fused into the butterflies.
//
// On B300 the FP64 pipe issues fused multiply-adds faster than separate adds
// or multiplies, and the FP64 passes are bound by that pipe.  A twiddled
// butterfly y+- = p +- w q costs 8 operations as a complex product followed
// by two complex additions; written in the tangent form of Goedecker
// (SIAM J. Sci. Comput. 18(6), 1997), w = c (1 + i tau) with tau = s / c,
//   t = q (1 + i tau)      2 FMAs
//   y+- = p +- c t         4 FMAs,
// it costs 6 FMAs (the cotangent form w = s (kappa + i), kappa = c / s, when
// |s| > |c|; 2 adds + 4 FMAs for the odd multiples of pi/4).  Every product
// and sum is still rounded once per operation, so each output component
// carries at most two roundings of a product-sum, as in the plain form.
//
// Structure: a size-R DFT is its first radix-2 layer, pairs (i, i + R/2),
// then dpost1<R>, the rest of the transform given that layer's results
// x[i] = a_i + a_{i+R/2} (P_i), x[i+R/2] = a_i - a_{i+R/2} (Q_i).  The
// stage-2 DFT of fft_pencil fuses the table twiddles into its first layer
// (fold_rt); the internal twiddles of the 16- and 32-point DFTs are folded
// into the first layer of their 4-point DFTs (fold_c).
// ---------------------------------------------------------------------------

// y+ = p + w q, y- = p - w q, w = exp(DIR 2 pi i m / 32), m a compile-time
// constant after unrolling (every branch but one folds away).
template <int DIR>
__device__ __forceinline__ void fold_c(double2 p, double2 q, int m, double2& yp, double2& ym) {
  m &= 31;
  if (m == 0) { yp = add<double>(p, q); ym = sub<double>(p, q); return; }
  if (m == 16) { yp = sub<double>(p, q); ym = add<double>(p, q); return; }
  if (m == 8) { yp = add_mul_i<double, DIR>(p, q); ym = sub_mul_i<double, DIR>(p, q); return; }
  if (m == 24) { yp = sub_mul_i<double, DIR>(p, q); ym = add_mul_i<double, DIR>(p, q); return; }
  const double c = cos32(m), sn = DIR * sin32(m);
  double2 t;
  double f;
  if ((m & 3) == 0 && (m & 7) != 0) {
    // odd multiple of pi/4: |c| = |s|, tau = s / c = +-1 exactly
    if ((c > 0) == (sn > 0)) t = mk<double>(q.x - q.y, q.y + q.x);   // tau = +1
    else t = mk<double>(q.x + q.y, q.y - q.x);                       // tau = -1
    f = c;
  } else if (fabs(c) >= fabs(sn)) {
    const double tau = sn / c;
    t = mk<double>(fma(-tau, q.y, q.x), fma(tau, q.x, q.y));
    f = c;
  } else {
    const double kap = c / sn;                                       // w = s (kappa + i)
    t = mk<double>(fma(kap, q.x, -q.y), fma(kap, q.y, q.x));
    f = sn;
  }
  yp = mk<double>(fma(f, t.x, p.x), fma(f, t.y, p.y));
  ym = mk<double>(fma(-f, t.x, p.x), fma(-f, t.y, p.y));
}

// The same with a table twiddle in tangent form: ct = (c, tau) of the
// forward factor w = c (1 + i tau); the inverse (DIR = +1) uses conj(w).
template <int DIR>
__device__ __forceinline__ void fold_rt(double2 p, double2 q, double2 ct, double2& yp, double2& ym) {
  const double tau = DIR < 0 ? ct.y : -ct.y;
  const double2 t = mk<double>(fma(-tau, q.y, q.x), fma(tau, q.x, q.y));
  yp = mk<double>(fma(ct.x, t.x, p.x), fma(ct.x, t.y, p.y));
  ym = mk<double>(fma(-ct.x, t.x, p.x), fma(-ct.x, t.y, p.y));
}

// The 4-point DFT given its first layer (P0, P1 | Q0, Q1) in x[0..3].
template <int DIR>
__device__ __forceinline__ void dpost1_4(double2& x0, double2& x1, double2& x2, double2& x3) {
  const double2 P0 = x0, P1 = x1, Q0 = x2, Q1 = x3;
  x0 = add<double>(P0, P1);
  x2 = sub<double>(P0, P1);
  x1 = add_mul_i<double, DIR>(Q0, Q1);
  x3 = sub_mul_i<double, DIR>(Q0, Q1);
}

template <int R, int DIR>
__device__ __forceinline__ void dpost1(double2 (&x)[R]) {
  if constexpr (R == 2) {
    // the first layer is the whole transform
  } else if constexpr (R == 4) {
    dpost1_4<DIR>(x[0], x[1], x[2], x[3]);
  } else if constexpr (R == 8) {
    // even half (a0, a2, a4, a6): first layer (P0, P2 | Q0, Q2); odd half
    // (a1, a3, a5, a7): (P1, P3 | Q1, Q3); then X_k, X_{k+4} = E_k +- w8^k O_k
    double2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    double2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    dpost1_4<DIR>(e0, e1, e2, e3);
    dpost1_4<DIR>(o0, o1, o2, o3);
    fold_c<DIR>(e0, o0, 0, x[0], x[4]);
    fold_c<DIR>(e1, o1, 4, x[1], x[5]);
    fold_c<DIR>(e2, o2, 8, x[2], x[6]);
    fold_c<DIR>(e3, o3, 12, x[3], x[7]);
  } else {
    // 16 = 4 x 4 and 32 = 8 x 4 (Cooley-Tukey, as dft_ab): A-point DFTs
    // over a_{b + 4a} (b = 0..3), internal twiddles w_R^{b k1}, 4-point DFTs
    // over b whose first layer takes the twiddles (fold_c).
    static_assert(R == 16 || R == 32, "FP64 register DFT sizes 2..32");
    constexpr int A = R / 4, H = R / 2, S = 32 / R;
    double2 T[4][A];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      // the first layer of the A-point DFT over a_{b + 4a} pairs a and a + A/2,
      // i.e. a_{b+4a} with a_{b+4a+H}: P_{b+4a} and Q_{b+4a}
      double2 t[A];
#pragma unroll
      for (int a = 0; a < A / 2; ++a) {
        t[a] = x[b + 4 * a];
        t[a + A / 2] = x[b + 4 * a + H];
      }
      dpost1<A, DIR>(t);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) T[b][k1] = t[k1];
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      double2 y[4];
      fold_c<DIR>(T[0][k1], T[2][k1], 2 * k1 * S, y[0], y[2]);
      const double2 p1 = mul_w32<double, DIR>(T[1][k1], k1 * S);
      fold_c<DIR>(p1, T[3][k1], 3 * k1 * S, y[1], y[3]);
      dpost1_4<DIR>(y[0], y[1], y[2], y[3]);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) x[k1 + A * k2] = y[k2];
    }
  }
}

template <int R, int DIR>
__device__ __forceinline__ void dftN_f64(double2 (&x)[R]) {
  if constexpr (R > 1) {
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      const double2 a = x[i], b = x[i + R / 2];
      x[i] = add<double>(a, b);
      x[i + R / 2] = sub<double>(a, b);
    }
    dpost1<R, DIR>(x);
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

// Host side of the FP64 stage table: entry of the factor w = c + i s
// (c = cos, s = -sin of 2 pi k1 t / L, already rounded to exact zeros where
// the exact value is zero).  Factors t < R2/2: (c, s).  Factors t >= R2/2:
// the tangent form (c, tau), tau = s / c, both rounded once from the long
// double values; at c = 0 (w = -+i) the pair (2^-600, s 2^600), whose
// product form c (1 + i tau) equals w to within 2^-600 relative (far below
// the rounding unit; no overflow for any finite float32-derived operand,
// which stays below 2^160 in magnitude).
inline double2 f64_stage_entry(long double c, long double s, bool tangent) {
  double2 r;
  if (!tangent) {
    r.x = (double)c;
    r.y = (double)s;
  } else if (c == 0.0L) {
    r.x = 0x1p-600;
    r.y = (double)(s * 0x1p600L);
  } else {
    r.x = (double)c;
    r.y = (double)(s / c);
  }
  return r;
}

// Pencils per tile of the strided passes: 64-byte rows (8 float32 or 4
// float64 complex values).
template <typename T> struct TileW { static constexpr int value = 16 / (int)sizeof(T) * 2; };

// The radix split of the two-stage schedule.  S = 0: stage 1 of size
// R1 = NT (V / NT DFTs per thread), stage 2 of size R2 = V (one per thread).
// S = 1, for odd log2 L (V = 2 NT): the sizes swapped -- stage 1 one DFT of
// size V on the thread's own values, stage 2 two DFTs of size NT -- with the
// same threads, registers and buffer (its exchange needs L + NT rows, less
// than the L + V of the natural-order exchanges).  Stage 1 runs R2 DFTs over
// x[n2 + R2 n1]; its output k1 of DFT n2 is twiddled by w^(n2 k1) and
// stage 2 runs the R1 DFTs over n2; output k1 + R1 k2 is X in natural order.
template <int L, int S>
struct Split {
  static_assert(S == 0 || (F2<L>::lg % 2 == 1), "the swapped split exists for odd log2 L");
  static constexpr int NT = F2<L>::NT, V = F2<L>::V;
  static constexpr int R1 = S ? V : NT;     // stage-1 DFT size
  static constexpr int R2 = S ? NT : V;     // stage-2 DFT size
  static constexpr int NB1 = R2 / NT;       // stage-1 DFTs per thread
  static constexpr int NB2 = R1 / NT;       // stage-2 DFTs per thread
};
// Host-side stage sizes of split S of L.
inline int split_r1(int L, int S) { return S ? L / f2_nt(L) : f2_nt(L); }
inline bool split_ok(int L, int S) { return S == 0 || (ilog2(L) % 2 == 1); }

// A thread's view of its pencil's column in the tile buffer (S: the radix
// split its transforms take).
template <typename T, int L, int W_, int S_ = 0>
struct Tile {
  static constexpr int W = W_;
  static constexpr int S = S_;
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
  using SP = Split<L, TL::S>;
  constexpr int R1 = SP::R1, R2 = SP::R2, NT = SP::NT, NB1 = SP::NB1, NB2 = SP::NB2, W = TL::W;
  tl.begin();
  v2<T>* buf = tl.buf();
#pragma unroll
  for (int b = 0; b < NB1; ++b) {
    v2<T> x[R1];
#pragma unroll
    for (int t = 0; t < R1; ++t) x[t] = v[b + t * NB1];
    dftN<R1, T, DIR>(x);
    // output t of stage-1 DFT n2 = j + b NT is element n2 R1 + t
    const int r0 = (j + b * NT) * (R1 + 1);
#pragma unroll
    for (int t = 0; t < R1; ++t) buf[(r0 + t) * W] = x[t];
  }
  TL::sync();
#pragma unroll
  for (int b = 0; b < NB2; ++b) {
    // stage-2 DFT k1 = j + b NT over n2 = t: element n2 R1 + k1 (row
    // t (R1 + 1) + k1), twiddled by w_L^{k1 t}; its output k2 is X[k1 + R1 k2],
    // the thread's natural-order value b + NB2 k2
    const int k1 = j + b * NT;
    v2<T> y[R2];
#pragma unroll
    for (int t = 0; t < R2; ++t) y[t] = buf[(t * (R1 + 1) + k1) * W];
    if constexpr (sizeof(T) == 4) {
      const float4* q = reinterpret_cast<const float4*>(tw) + k1;
#pragma unroll
      for (int i = 0; i < R2 / 2; ++i) {
        const float4 f = q[i * R1];   // factors 2i+1, 2i+2 of row k1
        y[2 * i + 1] = twmul<T, DIR>(y[2 * i + 1], mk<T>(f.x, f.y));
        if (2 * i + 2 < R2) y[2 * i + 2] = twmul<T, DIR>(y[2 * i + 2], mk<T>(f.z, f.w));
      }
      dftN<R2, T, DIR>(y);
    } else {
      // the stage-2 DFT's first layer, pairs (t, t + R2/2), with the table
      // twiddles fused in: factor t < R2/2 as a complex product, factor
      // t + R2/2 in tangent form (c, tau) folded into the butterfly
      constexpr int H = R2 / 2;
#pragma unroll
      for (int t = 0; t < H; ++t) {
        const v2<T> p = t == 0 ? y[0] : twmul<T, DIR>(y[t], tw[tw_index(R1, k1, t)]);
        fold_rt<DIR>(p, y[t + H], tw[tw_index(R1, k1, t + H)], y[t], y[t + H]);
      }
      dpost1<R2, DIR>(y);
    }
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[b + NB2 * k2] = y[k2];
  }
  tl.done();
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
