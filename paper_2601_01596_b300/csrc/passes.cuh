// passes.cuh -- the fused pass kernels of the correction loop (sm_103a).
//
// Storage.  A real item of shape (n0, .., n_{d-1}) (last axis x contiguous,
// Nx = 2M) keeps its spectrum "packed": rows of M complex values, one row
// per x-row of the field, so the spectrum has exactly as many scalars as the
// field.  Slot kx = 0 of each row holds X(kx=0) + i X(kx=M) of the x-R2C
// (both are real after the x transform).  The C2C transforms over the other
// axes are linear, so slot 0 then carries A + iB with A, B the spectra of
// the kx = 0 and kx = Nx/2 planes; A and B are Hermitian over the remaining
// axes and are separated (and clipped) only where the nonlinear f-clip needs
// them: A(k) = (C(k) + conj C(-k))/2, B(k) = (C(k) - conj C(-k))/(2i).
//
// Passes of one iteration (Alg. 1, Sec. IV-B; the loop body of Sec. IV-D):
//   3D: y-inverse, [x-inverse, s-clip, x-forward], y-forward,
//       [z-forward, check, f-clip, z-inverse]
//   2D: [x-inverse, s-clip, x-forward], [y-forward, check, f-clip, y-inverse]
// The check/clip pass ("chk") runs the outermost axis, after which the
// spectrum is complete; the s-clip pass ("px") runs the contiguous axis, the
// only place where e exists in registers.  Neither e nor the unclipped
// spectrum is written to HBM in steady state.
//
// Loop state lives on the device.  Every kernel reads its item's iteration
// counter t and picks its buffers by parity: the check at iteration t writes
// buffer t&1, the next iteration reads it and writes the other one, so the
// input of the last body (from which the returned iterate is rebuilt) is
// still intact when the loop stops.
#pragma once
#include <float.h>
#include <math.h>

#include <type_traits>

#include "fft_core.cuh"
#include "tma.cuh"

namespace ffcz {

struct ItemParams {
  double E, D, Es, Ds, thr, inv_n;   // bounds, shrunk bounds, stop threshold, 1/N
  float Esf, Dsf, thrf, inv_nf;      // the same in float32
  int64_t n;                         // points
  int32_t min_iters, max_iters;
  // 1D items (Bluestein): 1/(P N) and log2 P (0 for 2D/3D items)
  double inv_pn;
  float inv_pnf;
  int32_t logP;
  // factor on the FP64 rounding bound in the certification: 1, or for
  // pointwise bounds (where D = 1 and violations are ratios) 1 / min_k Delta_k
  double bscale;
  // spatial stopping threshold E(1 - eta/2) of the ADMM variant
  double thrs;
  float thrsf;
  int32_t pw;   // 1: pointwise bounds (E, D are 1; measures are ratios)
  int32_t h1;   // 1D, N even: certified through the N/2-point transform of x_2n + i x_2n+1
};

struct ItemState {
  unsigned long long vbits;      // max violation of the current check (double bits)
  unsigned long long emaxbits;   // max |e| (double bits)
  double sumsq;                  // sum e^2 (certification)
  unsigned long long act_s, act_f;
  unsigned long long last_act_s, last_act_f, prev_act_f;
  double f_ratio;                // last violation / D
  double v64, emax64, bound64;   // certification results
  int32_t t, done, status, preclip;
  int32_t certified, repairs, pad0, pad1;
  unsigned long long svbits;     // ADMM: max |a_t| of the loop's spatial check (double bits)
};

struct Group {
  int32_t ndim, Nz, Nmid, M;     // chk-axis length, middle-axis length (1 in 2D), Nx/2
  int64_t rows;                  // x-rows per item (N / Nx)
  const int32_t* item;           // global item index of each group member
  const int64_t* eoff;           // float offset of each member in e
  const int64_t* soff;           // complex offset of each member's spectrum
  const int64_t* coff;           // offset of each member's canonical half spectrum
  const int64_t* roff;           // offset of each member's first x-row among all items' rows
};

// Projection of the loop: Alg. 1 (POCS) or one of the variants that Sec. III
// names as alternatives (Dykstra; Douglas-Rachford on F' then S'; ADMM, which
// on F' then S' is Douglas-Rachford on S' then F').
enum Variant : int { PV_POCS = 0, PV_DYKSTRA = 1, PV_DR = 2, PV_ADMM = 3 };

enum Pred : int { P_ALL = 0, P_ACTIVE = 1, P_EXIT = 2, P_PRECLIP = 3, P_UNCERT = 4 };
enum Sel : int { S_CUR = 0, S_PREV = 1 };
enum Mode : int {
  M_CLIP = 1, M_MASK = 2, M_RECORD = 4, M_MEASURE = 8, M_PRECLIP = 16, M_NOWRITE = 32,
  M_CKPT = 64, M_COUNT = 128,
  M_ACC = 256   // exit x pass: add the result to e instead of storing it
};

struct Args {
  Group g;
  const ItemParams* prm;
  ItemState* st;
  void* B0;                // spectrum buffers (v2<T>)
  void* B1;
  float* e;                // spatial float32 buffer (in or out)
  const float* ein;        // separate float32 input (adjoint entry)
  uint32_t* mask;          // mask words (one per thread per pass)
  int64_t mask_thr;        // mask threads per group member (member gi's words start at gi mask_thr MW)
  int64_t mask_step;       // M_RECORD in the loop: words per iteration (the masks of iteration t at t mask_step)
  float* ckpt;             // checkpoint buffer for e_t
  int64_t ckpt_stride;     // floats per checkpoint (all items of the plan)
  int ckpt_every;
  int pred, sel_in, sel_out, mode;
  const void* tw;          // Stockham stage factors for the pass length
  const void* tw1;         // the same for the swapped radix split (Split<L, 1>; null if none)
  const void* twr;         // exp(-2 pi i k / Nx), k < M (x passes); exp(-2 pi i m / P) (1D)
  const void* bt;          // 1D: FFT of the wrapped chirp, [k1][k2] order, per item at soff
  const void* chirp;       // 1D: chirps b_n, n < N, per item at eoff
  int op1;                 // 1D pass operation (Op1)
  // 2D tensor maps of the float32 spectrum buffers for the TMA-fed passes,
  // two per group member ([2 gi + buffer]); null when the pass's buffers are
  // not the plan's float32 pair
  const CUtensorMap* tm_axis;
  const CUtensorMap* tm_chk;
  // the same view of the check pass's auxiliary packed field, one per group
  // member: the pointwise f-bounds (pw_f) or the projection variants'
  // residual (pv_r) (null: the check pass reads it with plain loads)
  const CUtensorMap* tm_aux;
  int* err;                // device error word (DevErr)
  // Alg. 1 edit recording (null: off).  ed_s: spatial edits, float32 laid
  // out like e.  Frequency edits in the packed spectrum layout: ed_f the
  // committed sum, ed_p the displacement of the latest f-clip of each slot,
  // ed_t 1 + the check index of that pending clip (0: none pending).
  float* ed_s;
  float2* ed_f;
  float2* ed_p;
  int* ed_t;
  // pointwise bounds (null: the item's scalar bounds): E_n laid out like e;
  // (Delta^Re, Delta^Im) in the packed spectrum layout (pw_f, slot kx of
  // each row for 1 <= kx < M) and, for the kx = 0 and Nx/2 planes, one
  // float4 (A bounds, B bounds) per row (pw_f0, at roff); with them the
  // item's E and D are 1 and the kernels compare and reduce ratios
  const float* pw_e;
  const float2* pw_f;
  const float4* pw_f0;
  // projection variant (Variant; float32 loops only).  pv_r: residual of the
  // frequency projection (Dykstra's p, Douglas-Rachford's z - P_F'(z)) in the
  // packed spectrum layout, read and rewritten in place by the check pass;
  // pv_q: Dykstra's q or ADMM's scaled dual u, float32 laid out like e, one
  // buffer per iteration parity (the exit pass rebuilds x_t from q_{t-1})
  int pv;
  float2* pv_r;
  float* pv_q[2];
  // first tile of a launch of the plain x and y passes (0: all rows), and
  // for the y pass the end of its tile range (0: all planes)
  int tile0;
  int tile1;
  // 1D certification of even lengths: 0 every member; 1 the N/2-point pass
  // of the members with h1 (the others return); 2 the N-point pass of the
  // members without h1.  zout: the N/2-point spectrum Z (float64, at the
  // member's spectrum offset)
  int half1;
  void* zout;
};

// Spatial edit of one complex register (two real points): S += (c - v).
// Each slot is touched by one thread per pass, so the add is a plain
// fire-and-forget reduction (no load on the thread's critical path) with
// the same result as a load, add and store.
template <typename T>
__device__ __forceinline__ void record_s(float2* at, T dx, T dy) {
  if (dx != T(0) || dy != T(0)) atomicAdd(at, make_float2((float)dx, (float)dy));
}

// Frequency edit of one packed slot clipped at check `t`: F += d.  Only a
// check whose violation is at most the stopping threshold can stop the loop
// (Alg. 1 projects nothing there), so a clip of a value above the threshold,
// or before min_iters, is final; a "marginal" clip also keeps d and 1 + t
// so that the edits pass after the loop can take it back if check t was the
// one that stopped.  Clips at the max_iters check are not recorded at all.
__device__ __forceinline__ void record_f(const Args& a, int64_t slot, float dx, float dy, int t,
                                         bool marginal) {
  if (dx == 0.f && dy == 0.f) return;
  atomicAdd(a.ed_f + slot, make_float2(dx, dy));   // one writer per slot and pass
  if (marginal) {
    a.ed_p[slot] = make_float2(dx, dy);
    a.ed_t[slot] = t + 1;
  }
}

__device__ __forceinline__ bool pred_ok(int pred, const ItemState& s, const ItemParams& p) {
  switch (pred) {
    case P_ACTIVE: return !s.done;
    case P_EXIT: return s.done && s.t >= 1;
    case P_PRECLIP: {
      // a non-finite field is left as it is: the check reports it
      const double em = __longlong_as_double((long long)s.emaxbits);
      return em > p.E && em <= DBL_MAX;
    }
    case P_UNCERT: return !s.certified;
    default: return true;
  }
}

template <typename T>
__device__ __forceinline__ v2<T>* pick(const Args& a, int sel, int t) {
  const int b = (sel == S_CUR) ? (t & 1) : ((t - 1) & 1);
  return reinterpret_cast<v2<T>*>(b ? a.B1 : a.B0);
}

// Per-tile launch geometry, shared by host and device.
template <typename T, int L, int W_ = TileW<T>::value>
struct Geo {
  static constexpr int W = W_;                         // pencils per tile
  static constexpr int NT = F2<L>::NT;                 // threads per pencil
  static constexpr int V = F2<L>::V;                   // values per thread
  static constexpr int TPT = NT * W;                   // threads per tile
  static constexpr int G = TPT >= 128 ? 1 : 128 / TPT; // tiles per CTA (>= 128 threads)
  static constexpr int NTHR = G * TPT;
  static constexpr int MW = (V + 7) / 8;               // mask words per thread
  // threads per SM the register budget is sized for: float32 with up to 8
  // values per thread 1024 (64 registers), 16 values 512 (128), 32 values
  // 384 (170); float64 512 (128) up to 8 values, else 256 (255)
  static constexpr int SMT = sizeof(T) == 4 ? (V >= 32 ? 384 : V >= 16 ? 512 : 1024) : (V >= 16 ? 256 : 512);
  static constexpr int MINB = SMT / NTHR > 0 ? SMT / NTHR : 1;
  // pointwise-bound variants hold the bounds of their values in registers too
  static constexpr int MINB_PW = MINB > 1 ? MINB - 1 : 1;
};

// Shared-memory carve-up: [G tile buffers][twiddles][R2C twiddles][reduction].
template <typename T, int L, int W = TileW<T>::value>
struct Smem {
  static constexpr size_t tiles = (size_t)Geo<T, L, W>::G * Tile<T, L, W>::ELEMS * sizeof(v2<T>);
  static constexpr size_t tw = (size_t)L * sizeof(v2<T>);
  static constexpr size_t twr = (size_t)L * sizeof(v2<T>);
  static constexpr size_t red = 32 * 8 * 3 + 32 * 4;
  static constexpr size_t bytes_axis = tiles + tw + red;
  static constexpr size_t bytes_x = tiles + tw + twr + red;
};

// Per-thread adjoint mask words: value u of the thread owns bits
// [PER (u % 8), PER (u % 8) + PER) of word u / 8 (PER = 2: Re, Im inside;
// PER = 4 on kx = 0 mirror tiles: Re A, Im A, Re B, Im B inside).
template <int MW>
struct MaskBits {
  uint32_t w[MW];
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int i = 0; i < MW; ++i) w[i] = 0u;
  }
  __device__ __forceinline__ void fill() {
#pragma unroll
    for (int i = 0; i < MW; ++i) w[i] = 0xffffffffu;
  }
  __device__ __forceinline__ void load(const uint32_t* m, int64_t thr) {
#pragma unroll
    for (int i = 0; i < MW; ++i) w[i] = m[thr * MW + i];
  }
  __device__ __forceinline__ void store(uint32_t* m, int64_t thr) const {
#pragma unroll
    for (int i = 0; i < MW; ++i) m[thr * MW + i] = w[i];
  }
  template <int PER>
  __device__ __forceinline__ uint32_t get(int u) const { return (w[u >> 3] >> (PER * (u & 7))) & ((1u << PER) - 1u); }
  template <int PER>
  __device__ __forceinline__ void put(int u, uint32_t b) { w[u >> 3] |= b << (PER * (u & 7)); }
};

// Block reduction of (max as non-negative double bits, count, sum).
struct Red {
  unsigned long long vbits;
  double sum;
  unsigned long long cnt;
};
__device__ __forceinline__ void block_reduce(Red& r, unsigned long long* sm) {
  const unsigned full = 0xffffffffu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r.vbits = max(r.vbits, __shfl_xor_sync(full, r.vbits, o));
    r.sum += __shfl_xor_sync(full, r.sum, o);
    r.cnt += __shfl_xor_sync(full, r.cnt, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  double* smd = reinterpret_cast<double*>(sm + 32);
  __syncthreads();
  if (lane == 0) { sm[wid] = r.vbits; smd[wid] = r.sum; sm[64 + wid] = r.cnt; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < nw; ++i) { r.vbits = max(r.vbits, sm[i]); r.sum += smd[i]; r.cnt += sm[64 + i]; }
  }
}

// Block reduction of a max (double bits) and, if `with_count`, a count.
__device__ __forceinline__ void block_max_count(unsigned long long& vb, unsigned long long& c,
                                                bool with_count, unsigned long long* sm) {
  const unsigned full = 0xffffffffu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    vb = max(vb, __shfl_xor_sync(full, vb, o));
    if (with_count) c += __shfl_xor_sync(full, c, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) { sm[wid] = vb; sm[64 + wid] = c; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < nw; ++i) { vb = max(vb, sm[i]); c += sm[64 + i]; }
  }
}

// Running max of |x|.  float32: one FMNMX per value (NaN is caught apart);
// float64: integer max of the magnitude bits (keeps the FP64 pipe for the
// butterflies; NaN orders above +inf).
template <typename T> struct AbsMax;
template <> struct AbsMax<float> {
  float m = 0.f;
  __device__ __forceinline__ void add(float x) { m = fmaxf(m, fabsf(x)); }
  __device__ __forceinline__ float val() const { return m; }
  __device__ __forceinline__ unsigned long long dbits(bool bad) const {
    return (unsigned long long)__double_as_longlong(bad ? (double)INFINITY : (double)m);
  }
};
template <> struct AbsMax<double> {
  unsigned long long b = 0;
  __device__ __forceinline__ void add(double x) {
    b = max(b, (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull);
  }
  __device__ __forceinline__ double val() const { return __longlong_as_double((long long)b); }
  __device__ __forceinline__ unsigned long long dbits(bool bad) const {
    return (bad || b > 0x7ff0000000000000ull) ? 0x7ff0000000000000ull : b;
  }
};

// A NaN or Inf anywhere in a field reaches every bin of the transform along
// each axis it passes (butterflies add it into every output, and Inf times an
// exact-zero twiddle component is NaN), so after the forward passes either the
// magnitude max is Inf or every value is NaN.  Two probes per thread detect
// the all-NaN case.
template <typename T, int V>
__device__ __forceinline__ bool nan_probe(const v2<T> (&v)[V]) {
  return (v[0].x != v[0].x) | (v[V - 1].y != v[V - 1].y);
}

// x / b for the normalised violations of pointwise bounds: float32 as x
// times the approximate reciprocal of PTX (rcp.approx.ftz.f32, within about
// one ulp of 1/b for the normal bounds the library accepts, FLT_MIN <= b;
// above 2^126 the reciprocal flushes to zero, so such a bin reads as inside
// unless |x| exceeds 2^126).  The ratio only decides when the float32 loop
// stops; the FP64 certification checks the bounds themselves.  A correctly
// rounded reciprocal, or one that keeps subnormals, is a multi-instruction
// sequence per value: at 512^3 it cost 0.16-0.19 ms per pass.
__device__ __forceinline__ float ratioT(float x, float b) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
  return x * r;
}
__device__ __forceinline__ double ratioT(double x, double b) { return x / b; }
// |x| / b for a measured maximum that a certification compares with 1: the
// approximate ratio, moved to the right side of 1 where it landed on the
// wrong one (|x| <= b is decided exactly)
__device__ __forceinline__ float ratio_cert(float x, float b) {
  const float ax = fabsf(x), r = ratioT(ax, b);
  return ax <= b ? fminf(r, 1.f) : fmaxf(r, 1.00000012f);
}

__device__ __forceinline__ float clampT(float x, float b) { return fminf(fmaxf(x, -b), b); }
__device__ __forceinline__ double clampT(double x, double b) { return fmin(fmax(x, -b), b); }

// Twiddle tables into shared memory: the length-L stage table and, for x
// passes, the M-entry R2C table; ends with a block barrier.
template <typename T>
__device__ __forceinline__ void load_tables(v2<T>* s_tw, const void* tw, int ntw, v2<T>* s_twr,
                                            const void* twr, int M) {
  const v2<T>* gtw = reinterpret_cast<const v2<T>*>(tw);
  for (int i = threadIdx.x; i < ntw; i += blockDim.x) s_tw[i] = gtw[i];
  if (s_twr) {
    const v2<T>* gtr = reinterpret_cast<const v2<T>*>(twr);
    for (int i = threadIdx.x; i < M; i += blockDim.x) s_twr[i] = gtr[i];
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// x passes: real rows <-> packed complex rows (R2C / C2R of length Nx = 2M
// through one length-M complex FFT of z[n] = r[2n] + i r[2n+1]).
// ---------------------------------------------------------------------------

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

// Exact binary32 -> binary64 widening by the IEEE 754 formats on the integer
// pipe (sign kept, exponent rebiased by 1023 - 127 = 896, the 23 fraction
// bits moved to the top of the 52), so that FP64 passes bound by the FP64
// pipe do not spend it on conversions.  Zero takes the same path; subnormal
// inputs, Inf and NaN (exponent field 0 with a nonzero fraction, or 255) use
// the hardware conversion.
__device__ __forceinline__ double widen_f32(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t ex = (b >> 23) & 0xffu, fr = b & 0x7fffffu, sg = b & 0x80000000u;
  if ((ex == 0u && fr != 0u) || ex == 0xffu) return (double)f;
  const uint32_t hi = (ex == 0u) ? sg : (sg | ((ex + 896u) << 20) | (fr >> 3));
  const uint32_t lo = (ex == 0u) ? 0u : (fr << 29);
  return __hiloint2double((int)hi, (int)lo);
}
template <typename T>
__device__ __forceinline__ T from_f32(float f) {
  if constexpr (sizeof(T) == 8) return widen_f32(f);
  else return f;
}

// The partner exchange of the R2C post- and C2R pre-processing without the
// tile buffer, for float32 tiles inside one warp: thread j of a pencil holds
// element j + NT u in v[u], and the partner M - k of k = j + NT u is element
// V - 1 - u of thread (NT - j) mod NT, or for j = 0 its own element
// (V - u) mod V.  The pairs (u, V - 1 - u) are exchanged together by
// register shuffles (half the shared-memory traffic of a store and a load),
// and f(k, x_k, x_{M-k}) gives the new value of element k.  Requires the
// tile's thread order tid = j W + w.
template <typename T, int M, class TL, class Fn>
__device__ __forceinline__ void pair_shfl(v2<T> (&v)[F2<M>::V], int j, Fn f) {
  constexpr int NT = F2<M>::NT, V = F2<M>::V, W = TL::W;
  static_assert(TL::TPT <= 32 && sizeof(T) == 4, "one-warp float32 tiles");
  const int lane = (int)(threadIdx.x & 31u);
  const int src = lane + (((NT - j) & (NT - 1)) - j) * W;
  const bool self = j == 0;
  v2<T> keep = v[0];   // thread j = 0: the previous step's element V - u, before its update
#pragma unroll
  for (int u = 0; u < V / 2; ++u) {
    constexpr unsigned FULL = 0xffffffffu;
    const int i = V - 1 - u;
    v2<T> mu, mi;   // x_{M-k} for k = j + NT u and for k = j + NT i
    mu.x = __shfl_sync(FULL, v[i].x, src);
    mu.y = __shfl_sync(FULL, v[i].y, src);
    mi.x = __shfl_sync(FULL, v[u].x, src);
    mi.y = __shfl_sync(FULL, v[u].y, src);
    if (self) {
      mu = keep;
      mi = v[u + 1];
    }
    keep = v[i];
    const v2<T> nu = f(j + NT * u, v[u], mu);
    const v2<T> ni = f(j + NT * i, v[i], mi);
    v[u] = nu;
    v[i] = ni;
  }
}

// Post-processing of Z = FFT_M(z) into the packed half spectrum P (in place
// in registers).  Each k needs Z[M-k], which another thread holds; it is
// read through one exchange in natural order (a warp barrier only, when the
// tile lies inside one warp).
// HALF = false leaves out the 1/2 of Fe and Fo: the result is 2 X, exact
// (a power of two), for the certification, which halves its maximum once.
template <typename T, int M, class TL, bool HALF = true>
__device__ __forceinline__ void r2c_post(v2<T> (&v)[F2<M>::V], int j, TL& tl,
                                         const v2<T>* __restrict__ twr) {
  constexpr int NT = F2<M>::NT, V = F2<M>::V;
  if constexpr (HALF && sizeof(T) == 4 && TL::TPT <= 32) {
    pair_shfl<T, M, TL>(v, j, [&](int k, v2<T> zk, v2<T> zm) {
      if (k == 0) return mk<T>(zk.x + zk.y, zk.x - zk.y);
      const v2<T> w = twr[k];
      const T ax = zk.x + zm.x, ay = zk.y - zm.y, bx = zk.x - zm.x, by = zk.y + zm.y;
      const T rx = fmaT(w.x, by, fmaT(w.y, bx, ax)), ry = fmaT(-w.x, bx, fmaT(w.y, by, ay));
      return mk<T>(T(0.5) * rx, T(0.5) * ry);
    });
    return;
  }
  store_nat<T, M, TL>(v, j, tl);
  if constexpr (!HALF) {
    // Paired form (certification): X(k) and X(M-k) share A, B and the
    // product Q = (W.x B.y + W.y B.x, W.y B.y - W.x B.x):
    // X(k) = A + Q, X(M-k) = conj(A - Q) (since W^(M-k) = -conj W^k), so the
    // threads holding k < M/2 compute both and hand X(M-k) over through the
    // tile buffer: 12 instead of 16 operations per pair.
    v2<T> xo[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int k = j + u * NT;
      const v2<T> zk = v[u];
      if (k == 0) {
        v[u] = mk<T>(T(2) * (zk.x + zk.y), T(2) * (zk.x - zk.y));
      } else if (2 * k <= M) {
        const v2<T> zm = tl.at(M - k);
        const v2<T> w = twr[k];
        const T ax = zk.x + zm.x, ay = zk.y - zm.y, bx = zk.x - zm.x, by = zk.y + zm.y;
        const T qx = fmaT(w.x, by, w.y * bx), qy = fmaT(-w.x, bx, w.y * by);
        v[u] = mk<T>(ax + qx, ay + qy);
        xo[u] = mk<T>(ax - qx, qy - ay);
      }
    }
    TL::sync();   // every read of Z is done
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int k = j + u * NT;
      if (k > 0 && 2 * k < M) tl.at(M - k) = xo[u];
    }
    TL::sync();
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int k = j + u * NT;
      if (2 * k > M) v[u] = tl.at(k);
    }
    tl.done();
    return;
  }
#pragma unroll
  for (int u = 0; u < V; ++u) {
    const int k = j + u * NT;
    const v2<T> zk = v[u];
    const v2<T> zm = tl.at((M - k) & (M - 1));
    if (k == 0) {
      v[u] = HALF ? mk<T>(zk.x + zk.y, zk.x - zk.y) : mk<T>(T(2) * (zk.x + zk.y), T(2) * (zk.x - zk.y));
    } else {
      // Fe = (Zk + conj Zm)/2, Fo = (Zk - conj Zm)/(2i), X = Fe + W^k Fo;
      // with A = Zk + conj Zm, B = Zk - conj Zm:
      // X = ((A.x + W.x B.y + W.y B.x) / 2, (A.y - W.x B.x + W.y B.y) / 2)
      const v2<T> w = twr[k];
      const T ax = zk.x + zm.x, ay = zk.y - zm.y, bx = zk.x - zm.x, by = zk.y + zm.y;
      const T rx = fmaT(w.x, by, fmaT(w.y, bx, ax)), ry = fmaT(-w.x, bx, fmaT(w.y, by, ay));
      v[u] = HALF ? mk<T>(T(0.5) * rx, T(0.5) * ry) : mk<T>(rx, ry);
    }
  }
  tl.done();
}

// Pre-processing of packed P into Z' = 2 Z so that IFFT_M(Z') / Nx gives
// the real row (P[M-k] read through one exchange as above).
template <typename T, int M, class TL>
__device__ __forceinline__ void c2r_pre(v2<T> (&v)[F2<M>::V], int j, TL& tl,
                                        const v2<T>* __restrict__ twr) {
  constexpr int NT = F2<M>::NT, V = F2<M>::V;
  if constexpr (sizeof(T) == 4 && TL::TPT <= 32) {
    pair_shfl<T, M, TL>(v, j, [&](int k, v2<T> xk, v2<T> xm) {
      if (k == 0) return mk<T>(xk.x + xk.y, xk.x - xk.y);
      const v2<T> w = twr[k];
      const T ax = xk.x + xm.x, ay = xk.y - xm.y, bx = xk.x - xm.x, by = xk.y + xm.y;
      return mk<T>(fmaT(-w.x, by, fmaT(w.y, bx, ax)), fmaT(w.x, bx, fmaT(w.y, by, ay)));
    });
    return;
  }
  store_nat<T, M, TL>(v, j, tl);
#pragma unroll
  for (int u = 0; u < V; ++u) {
    const int k = j + u * NT;
    const v2<T> xk = v[u];
    const v2<T> xm = tl.at((M - k) & (M - 1));
    if (k == 0) {
      v[u] = mk<T>(xk.x + xk.y, xk.x - xk.y);
    } else {
      // Z' = (Xk + conj Xm) + i (Xk - conj Xm) conj(W^k); with A, B as in
      // r2c_post: Z' = (A.x - W.x B.y + W.y B.x, A.y + W.x B.x + W.y B.y)
      const v2<T> w = twr[k];
      const T ax = xk.x + xm.x, ay = xk.y - xm.y, bx = xk.x - xm.x, by = xk.y + xm.y;
      v[u] = mk<T>(fmaT(-w.x, by, fmaT(w.y, bx, ax)), fmaT(w.x, bx, fmaT(w.y, by, ay)));
    }
  }
  tl.done();
}

#define FFCZ_X_PROLOGUE(T_, M_, W_, S_)                                           \
  using G_ = Geo<T_, M_, W_>;                                                     \
  using TL = Tile<T_, M_, W_, S_>;                                                \
  constexpr int V = G_::V;                                                        \
  extern __shared__ __align__(16) unsigned char smraw[];                          \
  v2<T_>* s_tiles = reinterpret_cast<v2<T_>*>(smraw);                            \
  v2<T_>* s_tw = s_tiles + G_::G * TL::ELEMS;                                     \
  v2<T_>* s_twr = s_tw + M_;                                                      \
  unsigned long long* s_red = reinterpret_cast<unsigned long long*>(s_twr + M_); \
  const int gi = by_;                                                             \
  const int item = a.g.item[gi];                                                  \
  const ItemParams& p = a.prm[item];                                              \
  ItemState& st = a.st[item];                                                     \
  if (!pred_ok(a.pred, st, p)) return;                                            \
  const int t_it = st.t;                                                          \
  const int g = threadIdx.x / G_::TPT, tid = threadIdx.x % G_::TPT;              \
  const int w = tid % G_::W, j = tid / G_::W;                                     \
  const int tile = a.tile0 + bx_ * G_::G + g;                                     \
  const int64_t prow = (int64_t)tile * G_::W + w;                                 \
  const bool live = prow < a.g.rows;                                              \
  const int64_t row = live ? prow : 0;                                            \
  const int64_t mthr = (int64_t)gi * a.mask_thr + (int64_t)tile * G_::TPT + tid;  \
  TL tl{s_tiles + g * TL::ELEMS + w, false};                                      \
  (void)t_it; (void)mthr;

// Entry / certification x pass: float32 real rows -> packed spectrum.
// PW: pointwise E_n (the measured maximum is max |e_n| / E_n).
// X2 (certification): the output is 2 X (see r2c_post).
template <typename T, int M, int W = TileW<T>::value, bool PW = false, bool X2 = false>
__device__ __forceinline__ void k_xfwd_body(const Args& a, const int bx_, const int by_) {
  FFCZ_X_PROLOGUE(T, M, W, 0)
  const float* src = (a.mode & M_MASK) ? a.ein : a.e;
  const float2* erow = reinterpret_cast<const float2*>(src + a.g.eoff[gi]) + row * M;
  float2* erow_w = reinterpret_cast<float2*>(a.e + a.g.eoff[gi]) + row * M;
  AbsMax<float> mx;
  float ssq = 0.f;
  unsigned long long cnt = 0;
  MaskBits<G_::MW> mb;
  mb.clear();
  if ((a.mode & M_MASK) && live) mb.load(a.mask, mthr);
  v2<T> v[V];
  bool bad = false;
  const float2* ebrow = PW ? reinterpret_cast<const float2*>(a.pw_e + a.g.eoff[gi]) + row * M : nullptr;
#pragma unroll
  for (int u = 0; u < V; ++u) {
    float2 x = erow[j + u * G_::NT];
    float2 eb = make_float2(1.f, 1.f);
    if constexpr (PW) eb = ebrow[j + u * G_::NT];
    if (a.mode & M_MEASURE) {
      if constexpr (PW) { mx.add(ratio_cert(x.x, eb.x)); mx.add(ratio_cert(x.y, eb.y)); }
      else { mx.add(x.x); mx.add(x.y); }
      bad |= (x.x != x.x) | (x.y != x.y);
      ssq = fmaf(x.x, x.x, fmaf(x.y, x.y, ssq));
    }
    if (a.mode & M_PRECLIP) {
      const float cx = PW ? clampT(x.x, p.Esf * eb.x) : clampT(x.x, p.Esf);
      const float cy = PW ? clampT(x.y, p.Esf * eb.y) : clampT(x.y, p.Esf);
      cnt += (cx != x.x) + (cy != x.y);
      if (a.ed_s && live)
        record_s<float>(reinterpret_cast<float2*>(a.ed_s + a.g.eoff[gi]) + row * M + j + u * G_::NT,
                        cx - x.x, cy - x.y);
      x.x = cx; x.y = cy;
      if (live) erow_w[j + u * G_::NT] = x;
    }
    if (a.mode & M_MASK) {
      const uint32_t b2 = mb.template get<2>(u);
      if (!(b2 & 1u)) x.x = 0.f;
      if (!(b2 & 2u)) x.y = 0.f;
    }
    v[u] = mk<T>(from_f32<T>(x.x), from_f32<T>(x.y));
  }
  load_tables<T>(s_tw, a.tw, M, s_twr, a.twr, M);
  fft_pencil<T, M, -1>(v, j, s_tw, tl);
  r2c_post<T, M, TL, !X2>(v, j, tl, s_twr);
  if (live) {
    v2<T>* out = pick<T>(a, a.sel_out, t_it) + a.g.soff[gi] + row * M;
#pragma unroll
    for (int u = 0; u < V; ++u) out[j + u * G_::NT] = v[u];
  }
  if (a.mode & (M_MEASURE | M_PRECLIP)) {
    // 2V float32 squares summed in float32: relative error < (2V+1) u32; the
    // bound that uses this sum takes (1 + 2^-17) of it (2V <= 64).
    Red r{live ? mx.dbits(bad) : 0ull, live ? (double)ssq * (1.0 + 0x1p-17) : 0.0, live ? cnt : 0ull};
    block_reduce(r, s_red);
    if (threadIdx.x == 0) {
      if (a.mode & M_MEASURE) {
        atomicMax(&st.emaxbits, r.vbits);
        atomicAdd(&st.sumsq, r.sum);
      }
      if ((a.mode & M_PRECLIP) && r.cnt) atomicAdd(&st.act_s, r.cnt);
    }
  }
}
template <typename T, int M, int W = TileW<T>::value, bool PW = false, bool X2 = false>
__global__ void __launch_bounds__(Geo<T, M, W>::NTHR, Geo<T, M, W>::MINB)
k_xfwd(Args a) {
  k_xfwd_body<T, M, W, PW, X2>(a, (int)blockIdx.x, (int)blockIdx.y);
}

// s-clip of the thread's values with every option (mask recording,
// checkpoint writes); the lean loop path clips without recording.
template <typename T, int V, int MW>
__device__ __forceinline__ void s_clip_full(v2<T> (&v)[V], T Es, bool count, MaskBits<MW>& mb,
                                            unsigned long long& cnt, float2* ck, int j, int NT) {
#pragma unroll
  for (int u = 0; u < V; ++u) {
    T x = v[u].x, y = v[u].y;
    const T cx = clampT(x, Es), cy = clampT(y, Es);
    const bool ix = (cx == x), iy = (cy == y);   // inside the s-cube
    if (count) cnt += (!ix) + (!iy);
    mb.template put<2>(u, (uint32_t)ix | ((uint32_t)iy << 1));
    v[u] = mk<T>(cx, cy);
    if (ck) ck[j + u * NT] = make_float2((float)cx, (float)cy);
  }
}

// Loop body x pass on one tile held in registers: C2R, scale 1/N, s-clip
// (or adjoint mask), R2C.  Returns the active-clip count of the thread.
// ED = false is the lean form of the forward loop: the edit recording, the
// adjoint mask modes and the checkpoints are compiled out.
template <typename T, int M, class TL, bool PW = false, bool ED = true, int PV = PV_POCS>
__device__ __forceinline__ unsigned long long px_core(const Args& a, const ItemParams& p, v2<T> (&v)[F2<M>::V],
                                                      int j, int64_t mthr, int64_t row, bool live,
                                                      int t_it, int64_t eoff, TL& tl, const v2<T>* twg,
                                                      const v2<T>* twr, float2* edrow = nullptr,
                                                      const float2* ebrow = nullptr,
                                                      const float2* qin = nullptr, float2* qout = nullptr,
                                                      AbsMax<T>* svm = nullptr) {
  constexpr int V = F2<M>::V, NT = F2<M>::NT, MW = (V + 7) / 8;
  float2 eb[PW ? V : 1];   // pointwise E_n of the thread's points, loaded before the transform
  if constexpr (PW) {
#pragma unroll
    for (int u = 0; u < V; ++u) eb[u] = ebrow[j + u * NT];
  }
  // Dykstra's q / ADMM's u of the previous iteration (zero before the
  // second s-projection), loaded before the transform
  constexpr bool QV = (PV == PV_DYKSTRA || PV == PV_ADMM);
  float2 qv[QV ? V : 1];
  if constexpr (QV) {
    const bool q_in = t_it >= 2 && live;
#pragma unroll
    for (int u = 0; u < V; ++u) qv[u] = q_in ? qin[j + u * NT] : make_float2(0.f, 0.f);
  }
  c2r_pre<T, M>(v, j, tl, twr);
  fft_pencil<T, M, +1>(v, j, twg, tl);
  unsigned long long cnt = 0;
  const T inv_n = sizeof(T) == 4 ? (T)p.inv_nf : (T)p.inv_n;
  const T Es = sizeof(T) == 4 ? (T)p.Esf : (T)p.Es;
  if constexpr (QV) {
    const bool count = (a.mode & M_COUNT) != 0;
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const T x = v[u].x * inv_n, y = v[u].y * inv_n;
      if constexpr (PV == PV_DYKSTRA) {
        // x' = P_S'(y + q), q <- y + q - x'
        const T wx = x + (T)qv[u].x, wy = y + (T)qv[u].y;
        const T cx = clampT(wx, Es), cy = clampT(wy, Es);
        if (count) cnt += (cx != wx) + (cy != wy);
        if (live) qout[j + u * NT] = make_float2((float)(wx - cx), (float)(wy - cy));
        v[u] = mk<T>(cx, cy);
      } else {
        // ADMM: a_t (the input) is checked against the s-cube; then
        // b = P_S'(a + u), u <- a + u - b, and the pass forwards b - u
        if (live) { svm->add(x); svm->add(y); }
        const T wx = x + (T)qv[u].x, wy = y + (T)qv[u].y;
        const T bx = clampT(wx, Es), by = clampT(wy, Es);
        if (count) cnt += (bx != wx) + (by != wy);
        const T ux = wx - bx, uy = wy - by;
        if (live) qout[j + u * NT] = make_float2((float)ux, (float)uy);
        v[u] = mk<T>(bx - ux, by - uy);
      }
    }
    fft_pencil<T, M, -1>(v, j, twg, tl);
    r2c_post<T, M>(v, j, tl, twr);
    return live ? cnt : 0ull;
  }
  AbsMax<T> mx;
#pragma unroll
  for (int u = 0; u < V; ++u) {
    v[u] = mk<T>(v[u].x * inv_n, v[u].y * inv_n);
    if constexpr (PW) {   // pointwise E_n: the vote runs on ratios
      mx.add(ratioT(v[u].x, (T)eb[u].x)); mx.add(ratioT(v[u].y, (T)eb[u].y));
    } else {
      mx.add(v[u].x); mx.add(v[u].y);
    }
  }
  const bool count = (a.mode & M_COUNT) != 0;
  const bool need_clip = __any_sync(0xffffffffu, mx.val() > Es);   // all lanes vote
  if (ED && (a.mode & M_MASK)) {
    MaskBits<MW> mb;
    mb.clear();
    if (live) mb.load(a.mask, mthr);
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const uint32_t b2 = mb.template get<2>(u);
      if (!(b2 & 1u)) v[u].x = T(0);
      if (!(b2 & 2u)) v[u].y = T(0);
    }
  } else if (ED && (a.mode & (M_RECORD | M_CKPT))) {
    // checkpoints of e_t for t = 0, m, 2m, ... below the item's K
    const bool ckn = (a.mode & M_CKPT) && a.ckpt_every > 0 && (t_it % a.ckpt_every) == 0 &&
                     t_it < p.max_iters && live;
    float2* ck = ckn ? reinterpret_cast<float2*>(a.ckpt + (int64_t)(t_it / a.ckpt_every) * a.ckpt_stride + eoff) +
                           row * M
                     : nullptr;
    MaskBits<MW> mb;
    mb.clear();
    s_clip_full<T, V, MW>(v, Es, count, mb, cnt, ck, j, NT);
    if ((a.mode & M_RECORD) && live) mb.store(a.mask + (int64_t)t_it * a.mask_step, mthr);
  } else if (need_clip) {
    // lean path: only warps holding a value outside the s-cube clip
    const bool rec_s = ED && edrow != nullptr && live;   // ED = false: the lean form
#pragma unroll
    for (int u = 0; u < V; ++u) {
      T bx = Es, by = Es;
      if constexpr (PW) { bx = Es * (T)eb[u].x; by = Es * (T)eb[u].y; }
      const T cx = clampT(v[u].x, bx), cy = clampT(v[u].y, by);
      if (count) cnt += (cx != v[u].x) + (cy != v[u].y);
      if (rec_s) record_s<T>(edrow + j + u * NT, cx - v[u].x, cy - v[u].y);   // spat_edits += eps' - eps
      v[u] = mk<T>(cx, cy);
    }
  }
  fft_pencil<T, M, -1>(v, j, twg, tl);
  r2c_post<T, M>(v, j, tl, twr);
  return live ? cnt : 0ull;
}

template <typename T, int M, int W = TileW<T>::value, bool PW = false, int PV = PV_POCS, bool FULL = true, int S = 0>
__device__ __forceinline__ void k_px_body(const Args& a, const int bx_, const int by_) {
  FFCZ_X_PROLOGUE(T, M, W, S)
  const v2<T>* in = pick<T>(a, a.sel_in, t_it) + a.g.soff[gi] + row * M;
  v2<T> v[V];
#pragma unroll
  for (int u = 0; u < V; ++u) v[u] = in[j + u * G_::NT];
  load_tables<T>(s_tw, S ? a.tw1 : a.tw, M, s_twr, a.twr, M);
  float2* edrow = a.ed_s ? reinterpret_cast<float2*>(a.ed_s + a.g.eoff[gi]) + row * M : nullptr;
  const float2* ebrow = PW ? reinterpret_cast<const float2*>(a.pw_e + a.g.eoff[gi]) + row * M : nullptr;
  const float2* qin = nullptr;
  float2* qout = nullptr;
  if constexpr (PV != PV_POCS) {
    qin = reinterpret_cast<const float2*>(a.pv_q[(t_it - 1) & 1] + a.g.eoff[gi]) + row * M;
    qout = reinterpret_cast<float2*>(a.pv_q[t_it & 1] + a.g.eoff[gi]) + row * M;
  }
  AbsMax<T> svm;
  unsigned long long cnt = px_core<T, M, TL, PW, FULL, PV>(a, p, v, j, mthr, row, live, t_it, a.g.eoff[gi], tl,
                                                           s_tw, s_twr, edrow, ebrow, qin, qout, &svm);
  if (live) {
    v2<T>* out = pick<T>(a, a.sel_out, t_it) + a.g.soff[gi] + row * M;
#pragma unroll
    for (int u = 0; u < V; ++u) out[j + u * G_::NT] = v[u];
  }
  if constexpr (PV == PV_ADMM) {
    // spatial check of a_t: block max, one atomic per CTA (NaN -> +inf)
    unsigned long long vb = live ? svm.dbits(svm.val() != svm.val()) : 0ull, cz = 0ull;
    block_max_count(vb, cz, false, s_red);
    if (threadIdx.x == 0) atomicMax(&st.svbits, vb);
  }
  if (a.mode & M_COUNT) {
    Red r{0ull, 0.0, cnt};
    block_reduce(r, s_red);
    if (threadIdx.x == 0 && r.cnt) atomicAdd(&st.act_s, r.cnt);
  }
}
template <typename T, int M, int W = TileW<T>::value, bool PW = false, int PV = PV_POCS, bool FULL = true, int S = 0>
__global__ void __launch_bounds__(Geo<T, M, W>::NTHR,
                                  (PW || PV != PV_POCS) ? Geo<T, M, W>::MINB_PW : Geo<T, M, W>::MINB)
k_px(Args a) {
  k_px_body<T, M, W, PW, PV, FULL, S>(a, (int)blockIdx.x, (int)blockIdx.y);
}

// Exit epilogue of one row (after the C2R): scale 1/N, (Dykstra) + q_{t-1},
// s-clip when M_CLIP (again after rounding to float32), store or (M_ACC)
// add to e.
template <typename T, int V, bool PW, int PV>
// ebr / qr: the thread's E_n / Dykstra q loaded before the transform
// (null: read from ebrow / qrow here).
__device__ __forceinline__ void xexit_store(const Args& a, const ItemParams& p, v2<T> (&v)[V], int j, int NT,
                                            float2* erow, const float2* ebrow, const float2* qrow,
                                            const float2* ebr = nullptr, const float2* qr = nullptr) {
  const T inv_n = sizeof(T) == 4 ? (T)p.inv_nf : (T)p.inv_n;
  const T Es = sizeof(T) == 4 ? (T)p.Esf : (T)p.Es;
#pragma unroll
  for (int u = 0; u < V; ++u) {
    T x = v[u].x * inv_n, y = v[u].y * inv_n;
    if (PV == PV_DYKSTRA && qrow) {
      const float2 q = qr ? qr[u] : qrow[j + u * NT];
      x += (T)q.x;
      y += (T)q.y;
    }
    float2 eb = make_float2(1.f, 1.f);
    if constexpr (PW) eb = ebr ? ebr[u] : ebrow[j + u * NT];
    if (a.mode & M_CLIP) {
      if constexpr (PW) { x = clampT(x, Es * (T)eb.x); y = clampT(y, Es * (T)eb.y); }
      else { x = clampT(x, Es); y = clampT(y, Es); }
    }
    float fx = (float)x, fy = (float)y;
    if (a.mode & M_CLIP) {
      // keep the float32 result inside the shrunk cube after rounding
      if constexpr (PW) { fx = clampT(fx, p.Esf * eb.x); fy = clampT(fy, p.Esf * eb.y); }
      else { fx = clampT(fx, p.Esf); fy = clampT(fy, p.Esf); }
    }
    if (a.mode & M_ACC) {
      const float2 o = erow[j + u * NT];
      fx += o.x; fy += o.y;
    }
    erow[j + u * NT] = make_float2(fx, fy);
  }
}

// Exit x pass: C2R, scale 1/N, s-clip, store float32 e (rebuilds the iterate
// e_t from the input of the last loop body).  In mask mode (adjoint exit)
// no clip is applied.
template <typename T, int M, int W = TileW<T>::value, bool PW = false, int PV = PV_POCS>
__device__ __forceinline__ void k_xexit_body(const Args& a, const int bx_, const int by_) {
  FFCZ_X_PROLOGUE(T, M, W, 0)
  const v2<T>* in = pick<T>(a, a.sel_in, t_it) + a.g.soff[gi] + row * M;
  v2<T> v[V];
#pragma unroll
  for (int u = 0; u < V; ++u) v[u] = in[j + u * G_::NT];
  // pointwise E_n of the thread's points, loaded before the transform
  const float2* ebrow = PW ? reinterpret_cast<const float2*>(a.pw_e + a.g.eoff[gi]) + row * M : nullptr;
  float2 ebr[PW ? V : 1];
  if constexpr (PW) {
#pragma unroll
    for (int u = 0; u < V; ++u) ebr[u] = ebrow[j + u * G_::NT];
  }
  // Dykstra: x_t = P_S'(y_{t-1} + q_{t-1}) (q_0 = 0); q loaded before the
  // transform too
  const float2* qrow = (PV == PV_DYKSTRA && t_it >= 2)
                           ? reinterpret_cast<const float2*>(a.pv_q[(t_it - 1) & 1] + a.g.eoff[gi]) + row * M
                           : nullptr;
  float2 qr[PV == PV_DYKSTRA ? V : 1];
  if constexpr (PV == PV_DYKSTRA) {
    if (qrow) {
#pragma unroll
      for (int u = 0; u < V; ++u) qr[u] = qrow[j + u * G_::NT];
    }
  }
  load_tables<T>(s_tw, a.tw, M, s_twr, a.twr, M);
  c2r_pre<T, M>(v, j, tl, s_twr);
  fft_pencil<T, M, +1>(v, j, s_tw, tl);
  float2* erow = reinterpret_cast<float2*>(a.e + a.g.eoff[gi]) + row * M;
  if (live)
    xexit_store<T, V, PW, PV>(a, p, v, j, G_::NT, erow, ebrow, qrow, PW ? ebr : nullptr,
                              PV == PV_DYKSTRA ? qr : nullptr);
}
template <typename T, int M, int W = TileW<T>::value, bool PW = false, int PV = PV_POCS>
__global__ void __launch_bounds__(Geo<T, M, W>::NTHR, Geo<T, M, W>::MINB)
k_xexit(Args a) {
  k_xexit_body<T, M, W, PW, PV>(a, (int)blockIdx.x, (int)blockIdx.y);
}
// ---------------------------------------------------------------------------
// Strided axis passes
// ---------------------------------------------------------------------------

#define FFCZ_AXIS_PROLOGUE(T_, L_, W_, S_)                                        \
  using G_ = Geo<T_, L_, W_>;                                                     \
  using TL = Tile<T_, L_, W_, S_>;                                                \
  constexpr int V = G_::V;                                                        \
  extern __shared__ __align__(16) unsigned char smraw[];                          \
  v2<T_>* s_tiles = reinterpret_cast<v2<T_>*>(smraw);                            \
  v2<T_>* s_tw = s_tiles + G_::G * TL::ELEMS;                                     \
  unsigned long long* s_red = reinterpret_cast<unsigned long long*>(s_tw + L_);  \
  (void)s_red;                                                                    \
  const int gi = by_;                                                             \
  const int item = a.g.item[gi];                                                  \
  const ItemParams& p = a.prm[item];                                              \
  ItemState& st = a.st[item];                                                     \
  if (!pred_ok(a.pred, st, p)) return;                                            \
  const int t_it = st.t;                                                          \
  const int g = threadIdx.x / G_::TPT, tid = threadIdx.x % G_::TPT;              \
  const int w = tid % G_::W, j = tid / G_::W;                                     \
  const int tile = a.tile0 + bx_ * G_::G + g;                                     \
  const int64_t mthr = (int64_t)gi * a.mask_thr + (int64_t)tile * G_::TPT + tid;  \
  TL tl{s_tiles + g * TL::ELEMS + w, false};                                      \
  (void)mthr;

// Plain C2C along the middle axis of a 3D item (y): pencils at fixed (z, kx).
template <typename T, int L, int DIR, int W = TileW<T>::value, int S = 0>
__device__ __forceinline__ void k_axis_body(const Args& a, const int bx_, const int by_) {
  FFCZ_AXIS_PROLOGUE(T, L, W, S)
  const int M = a.g.M;
  const unsigned tpr = (unsigned)(M / G_::W);     // tiles per z-plane
  const int ntiles = a.tile1 ? a.tile1 : a.g.Nz * (int)tpr;
  const bool live = tile < ntiles;
  const int z = live ? (int)((unsigned)tile / tpr) : 0;
  const int kx = live ? (int)((unsigned)tile % tpr) * G_::W + w : 0;
  const int64_t off = (int64_t)z * L * M + kx;

  const int64_t ustride = (int64_t)G_::NT * M;
  const v2<T>* in = pick<T>(a, a.sel_in, t_it) + a.g.soff[gi] + off + (int64_t)j * M;
  v2<T> v[V];
#pragma unroll
  for (int u = 0; u < V; ++u) v[u] = in[u * ustride];
  load_tables<T>(s_tw, S ? a.tw1 : a.tw, L, nullptr, nullptr, 0);   // overlaps the loads
  fft_pencil<T, L, DIR>(v, j, s_tw, tl);
  if (live) {
    v2<T>* out = pick<T>(a, a.sel_out, t_it) + a.g.soff[gi] + off + (int64_t)j * M;
#pragma unroll
    for (int u = 0; u < V; ++u) out[u * ustride] = v[u];
  }
}
template <typename T, int L, int DIR, int W = TileW<T>::value, int S = 0>
__global__ void __launch_bounds__(Geo<T, L, W>::NTHR, Geo<T, L, W>::MINB)
k_axis(Args a) {
  k_axis_body<T, L, DIR, W, S>(a, (int)blockIdx.x, (int)blockIdx.y);
}

// Check / f-clip pass along the outermost axis (z in 3D, y in 2D): forward
// FFT completes the spectrum; the violation max over all bins is reduced
// (CheckConvergence), Re and Im are clipped to +-D' (ProjectOntoFCube), and
// the inverse FFT of this axis is applied before the store.
//
// Tiles are of two kinds.  Main tiles: W consecutive kx at one middle index
// (slot kx = 0 skipped).  Mirror tiles: the kx = 0 pencils, in pairs (m, -m)
// of middle indices so that A and B can be separated; a pencil that is its
// own mirror (m = 0 or Nmid/2) fills both slots of its pair and only the
// first slot stores.
struct ChkTile {
  int off;       // complex offset of the pencil in the item's spectrum
  bool owner;    // this slot stores its pencil
  bool valid;    // this slot holds bins to check
  bool mirror;   // the tile is a kx = 0 mirror tile
  bool live;
};

template <int W>
__device__ __forceinline__ ChkTile chk_decode(int tile, int w, int M, int Nmid) {
  ChkTile c{0, false, false, false, false};
  const unsigned tpr = (unsigned)(M / W);
  const int nmain = Nmid * (int)tpr;
  const int npairs = Nmid / 2 + 1;   // pairs (m, -m), m = 0..Nmid/2
  const int nmirror = (npairs + W / 2 - 1) / (W / 2);
  c.live = tile < nmain + nmirror;
  c.mirror = c.live && tile >= nmain;
  if (c.live && !c.mirror) {
    const int mid = (int)((unsigned)tile / tpr);
    const int kx = (int)((unsigned)tile % tpr) * W + w;
    c.off = mid * M + kx;
    c.valid = kx != 0;
    c.owner = c.valid;
  } else if (c.mirror) {
    const int q = (tile - nmain) * (W / 2) + (w >> 1);
    const int m = w & 1;
    const int nh = Nmid / 2;
    c.valid = q < npairs;
    const bool selfm = (q == 0) || (q == nh);
    const int mid = !c.valid ? 0 : (selfm ? q : (m ? Nmid - q : q));
    c.off = mid * M;
    c.owner = c.valid && (m == 0 || !selfm);
  }
  return c;
}

__host__ __device__ inline int chk_ntiles(int W, int M, int Nmid) {
  const int npairs = Nmid / 2 + 1;
  return Nmid * (M / W) + (npairs + W / 2 - 1) / (W / 2);
}

// Everything of the check pass between load and store for one tile in
// registers.  cta_has_mirror must be uniform over the CTA.
// Pointwise bounds of a check-pass pencil: its packed slots (step estride
// per kz) or, on a mirror tile, the per-row float4 of the kx = 0 and Nx/2
// planes (viewed as float2 pairs: A bounds, then B bounds).
__device__ __forceinline__ void pw_pencil(const Args& a, int gi, const ChkTile& c, int M, int Nmid,
                                          int64_t estride, const float2*& pwb, int64_t& pws) {
  if (c.mirror) {
    pwb = reinterpret_cast<const float2*>(a.pw_f0 + a.g.roff[gi] + c.off / M);
    pws = 2 * (int64_t)Nmid;
  } else {
    pwb = a.pw_f + a.g.soff[gi] + c.off;
    pws = estride;
  }
}

// Source of the pointwise bounds in chk_core: by default they are read from
// global memory into registers before the forward transform; a caller that
// stages them in shared memory passes a functor with late = true, called
// after the forward transform, which waits until the staged bounds landed.
struct QEarly {
  static constexpr bool late = false;
  uint32_t sq = 0;
  __device__ __forceinline__ void operator()() const {}
};

// FULL = false compiles out the adjoint mask modes and the edit recording
// (the forward loop's lean variant: less code, no mask-bit bookkeeping).
template <typename T, int L, class TL, bool PW = false, int PV = PV_POCS, bool FULL = true, class QW = QEarly>
__device__ __forceinline__ void chk_core(const Args& a, const ItemParams& p, ItemState& st,
                                         v2<T> (&v)[F2<L>::V], int j, int w, int64_t mthr,
                                         const ChkTile& c, bool cta_has_mirror, TL& tl,
                                         const v2<T>* twg, unsigned long long* s_red,
                                         unsigned long long* acc_vb = nullptr,
                                         unsigned long long* acc_cnt = nullptr,
                                         int64_t ed_slot0 = 0, int64_t ed_ustride = 0, int t_chk = 0,
                                         const float2* pwb = nullptr, int64_t pws = 0, int pwM = 0,
                                         QW qwait = QW{}) {
  // pwb: pointwise (Delta^Re, Delta^Im) of this pencil's bin at kz = 0, pws
  // the step per kz; on mirror tiles pwb holds the bounds of A and pwb + pwM
  // those of B
  constexpr int NT = F2<L>::NT, V = F2<L>::V, MW = (V + 7) / 8;
  // pointwise bounds of the thread's bins, loaded before the forward
  // transform so that their latency hides behind it (or, staged in shared
  // memory, read where they are used)
  constexpr bool QLATE = PW && QW::late;
  float2 qb[(PW && !QLATE) ? V : 1];
  if constexpr (PW && !QLATE) {
#pragma unroll
    for (int u = 0; u < V; ++u) qb[u] = pwb[(int64_t)(j + u * NT) * pws];
  }
  // bounds of value u: qbound on the mirror path (any tile), qmain where
  // only main tiles' results are kept (staged: a shared-memory read at a
  // compile-time offset, whatever the tile)
  auto qbound = [&](int u) -> float2 {
    if constexpr (QLATE) return pwb[(int64_t)(j + u * NT) * pws];
    else return qb[PW ? u : 0];
  };
  auto qmain = [&](int u) -> float2 {
    if constexpr (QLATE) {
      float2 q;
      asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];"
                   : "=f"(q.x), "=f"(q.y)
                   : "r"(qwait.sq + (uint32_t)((j + u * NT) * TL::W) * 8u));
      return q;
    } else {
      return qb[PW ? u : 0];
    }
  };
  // Dykstra / Douglas-Rachford: the residual r of the previous frequency
  // projection (zero before the first one), loaded before the transform
  constexpr bool RES = (PV == PV_DYKSTRA || PV == PV_DR);
  constexpr bool RLATE = RES && QW::late;   // residual staged in shared memory
  const bool res_in = RES && t_chk >= 1 && c.valid;
  // residual of value u: rr_any on the mirror path (a global load when
  // staged), rr_main where only main tiles' results are kept
  float2 rr[(RES && !RLATE) ? V : 1];
  auto rr_any = [&](int u) -> float2 {
    if constexpr (RLATE) return res_in ? a.pv_r[ed_slot0 + u * ed_ustride] : make_float2(0.f, 0.f);
    else return rr[RES ? u : 0];
  };
  auto rr_main = [&](int u) -> float2 {
    if constexpr (RLATE) {
      float2 r;
      asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];"
                   : "=f"(r.x), "=f"(r.y)
                   : "r"(qwait.sq + (uint32_t)((j + u * NT) * TL::W) * 8u));
      return res_in ? r : make_float2(0.f, 0.f);
    } else {
      return rr[RES ? u : 0];
    }
  };
  if constexpr (RES && !RLATE) {
#pragma unroll
    for (int u = 0; u < V; ++u) rr[u] = res_in ? a.pv_r[ed_slot0 + u * ed_ustride] : make_float2(0.f, 0.f);
  }
  fft_pencil<T, L, -1>(v, j, twg, tl);
  if constexpr (QW::late) qwait();
  const T Ds = sizeof(T) == 4 ? (T)p.Dsf : (T)p.Ds;
  AbsMax<T> mx;
  bool bad = false;
  unsigned long long cnt = 0;
  MaskBits<MW> mb;
  mb.clear();
  const bool rec = FULL && (a.mode & M_RECORD) != 0, use_mask = FULL && (a.mode & M_MASK) != 0;
  const bool clip = (a.mode & M_CLIP) != 0, count = (a.mode & M_COUNT) != 0;
  // freq_edits += delta' - delta (not at the max_iters check, which stops)
  const bool rec_f = FULL && clip && a.ed_t != nullptr && c.owner && t_chk < p.max_iters;
  const bool may_stop = t_chk >= p.min_iters;
  const T thr = sizeof(T) == 4 ? (T)p.thrf : (T)p.thr;
  if (use_mask && c.live) mb.load(a.mask, mthr);
  if constexpr (RES) {
    if (cta_has_mirror) {
      // check on x's spectrum C (A, B separated), then the projection of
      // C' = C + r, whose partner values need a second exchange
      store_nat<T, L, TL>(v, j, tl);
      if (c.mirror) {
        const int dw = (w ^ 1) - w;
#pragma unroll
        for (int u = 0; u < V; ++u) {
          const v2<T> cc = v[u], m = tl.at_other((L - (j + u * NT)) & (L - 1), dw);
          const T ar = T(0.5) * (cc.x + m.x), ai = T(0.5) * (cc.y - m.y);
          const T br = T(0.5) * (cc.y + m.y), bi = T(0.5) * (m.x - cc.x);
          if (c.valid) { mx.add(ar); mx.add(ai); mx.add(br); mx.add(bi); }
          bad |= c.valid && ((ar != ar) | (ai != ai) | (br != br) | (bi != bi));
        }
      }
      tl.done();
      if (c.mirror) {
#pragma unroll
        for (int u = 0; u < V; ++u) {
          const float2 r = rr_any(u);
          v[u] = mk<T>(v[u].x + (T)r.x, v[u].y + (T)r.y);
        }
      }
      store_nat<T, L, TL>(v, j, tl);
      if (c.mirror) {
        const int dw = (w ^ 1) - w;
#pragma unroll
        for (int u = 0; u < V; ++u) {
          const v2<T> cc = v[u], m = tl.at_other((L - (j + u * NT)) & (L - 1), dw);
          const T ar = T(0.5) * (cc.x + m.x), ai = T(0.5) * (cc.y - m.y);
          const T br = T(0.5) * (cc.y + m.y), bi = T(0.5) * (m.x - cc.x);
          const T car = clampT(ar, Ds), cai = clampT(ai, Ds), cbr = clampT(br, Ds), cbi = clampT(bi, Ds);
          if (c.owner && count) cnt += (car != ar) + (cai != ai) + (cbr != br) + (cbi != bi);
          const T yx = car - cbi, yy = cai + cbr;          // Y = A' + i B'
          const T rx = cc.x - yx, ry = cc.y - yy;          // r <- C' - Y
          if (c.owner) a.pv_r[ed_slot0 + u * ed_ustride] = make_float2((float)rx, (float)ry);
          v[u] = PV == PV_DYKSTRA ? mk<T>(yx, yy) : mk<T>(yx - rx, yy - ry);
        }
      }
      tl.done();
    }
  } else if (cta_has_mirror) {
    store_nat<T, L, TL>(v, j, tl);
    if (c.mirror) {
      const int dw = (w ^ 1) - w;
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const v2<T> cc = v[u], m = tl.at_other((L - (j + u * NT)) & (L - 1), dw);
        // A = (C + conj Cm)/2, B = (C - conj Cm)/(2i)
        T ar = T(0.5) * (cc.x + m.x), ai = T(0.5) * (cc.y - m.y);
        T br = T(0.5) * (cc.y + m.y), bi = T(0.5) * (m.x - cc.x);
        T bar = T(1), bai = T(1), bbr = T(1), bbi = T(1);   // pointwise bounds (ratios)
        if constexpr (PW) {
          const float2 qB = pwb[(int64_t)(j + u * NT) * pws + pwM];
          const float2 qA = qbound(u);
          bar = (T)qA.x; bai = (T)qA.y; bbr = (T)qB.x; bbi = (T)qB.y;
        }
        if (c.valid) {
          if constexpr (PW) { mx.add(ratioT(ar, bar)); mx.add(ratioT(ai, bai)); mx.add(ratioT(br, bbr)); mx.add(ratioT(bi, bbi)); }
          else { mx.add(ar); mx.add(ai); mx.add(br); mx.add(bi); }
        }
        bad |= c.valid && ((ar != ar) | (ai != ai) | (br != br) | (bi != bi));
        if (clip) {
          const T car = clampT(ar, PW ? Ds * bar : Ds), cai = clampT(ai, PW ? Ds * bai : Ds);
          const T cbr = clampT(br, PW ? Ds * bbr : Ds), cbi = clampT(bi, PW ? Ds * bbi : Ds);
          const bool iar = car == ar, iai = cai == ai, ibr = cbr == br, ibi = cbi == bi;
          if (c.owner) cnt += (!iar) + (!iai) + (!ibr) + (!ibi);
          if (FULL)
            mb.template put<4>(u, (uint32_t)iar | ((uint32_t)iai << 1) | ((uint32_t)ibr << 2) |
                                      ((uint32_t)ibi << 3));
          ar = car; ai = cai; br = cbr; bi = cbi;
          if (rec_f) {
            const T nx = ar - bi, ny = ai + br;
            T big = fmax(fmax(fabs(T(0.5) * (cc.x + m.x)), fabs(T(0.5) * (cc.y - m.y))),
                         fmax(fabs(T(0.5) * (cc.y + m.y)), fabs(T(0.5) * (m.x - cc.x))));
            if constexpr (PW)
              big = fmax(fmax(ratioT(fabs(T(0.5) * (cc.x + m.x)), bar), ratioT(fabs(T(0.5) * (cc.y - m.y)), bai)),
                         fmax(ratioT(fabs(T(0.5) * (cc.y + m.y)), bbr), ratioT(fabs(T(0.5) * (m.x - cc.x)), bbi)));
            record_f(a, ed_slot0 + u * ed_ustride, (float)(nx - cc.x), (float)(ny - cc.y), t_chk,
                     may_stop && big <= thr);
          }
        } else if (use_mask) {
          const uint32_t b4 = mb.template get<4>(u);
          if (!(b4 & 1u)) ar = T(0);
          if (!(b4 & 2u)) ai = T(0);
          if (!(b4 & 4u)) br = T(0);
          if (!(b4 & 8u)) bi = T(0);
        }
        v[u] = mk<T>(ar - bi, ai + br);   // C' = A' + i B'
      }
    }
    tl.done();
  }
  // Main-tile magnitude max, and one vote over all lanes (a warp can span
  // several tiles when tiles are small, so the vote is outside any branch
  // that depends on the tile).
  AbsMax<T> tm;
#pragma unroll
  for (int u = 0; u < V; ++u) {
    if constexpr (PW) {
      const float2 q = qmain(u);
      tm.add(ratioT(v[u].x, (T)q.x)); tm.add(ratioT(v[u].y, (T)q.y));
    }
    else { tm.add(v[u].x); tm.add(v[u].y); }
  }
  const bool need_clip = __any_sync(0xffffffffu, !c.mirror && tm.val() > Ds);
  if (RES && !c.mirror) {
    if (c.valid) { mx = tm; bad = nan_probe<T, V>(v); }
    // y = P_F'(x + r), r <- x + r - y; output y (Dykstra) or 2y - (x + r) =
    // y - r (Douglas-Rachford)
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const float2 r = rr_main(u);
      const T x = v[u].x + (T)r.x, y = v[u].y + (T)r.y;
      const T cx = clampT(x, Ds), cy = clampT(y, Ds);
      if (count && c.owner) cnt += 2 * ((cx != x) + (cy != y));
      const T rx = x - cx, ry = y - cy;
      if (c.owner) a.pv_r[ed_slot0 + u * ed_ustride] = make_float2((float)rx, (float)ry);
      v[u] = PV == PV_DYKSTRA ? mk<T>(cx, cy) : mk<T>(cx - rx, cy - ry);
    }
  } else if (!c.mirror) {
    if (c.valid) { mx = tm; bad = nan_probe<T, V>(v); }
    if (use_mask) {
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const uint32_t b2 = mb.template get<2>(u);
        if (!(b2 & 1u)) v[u].x = T(0);
        if (!(b2 & 2u)) v[u].y = T(0);
      }
    } else if (clip && (rec || need_clip)) {
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const T x = v[u].x, y = v[u].y;
        T qx = T(1), qy = T(1);
        if constexpr (PW) { const float2 q = qmain(u); qx = (T)q.x; qy = (T)q.y; }
        const T cx = clampT(x, PW ? Ds * qx : Ds), cy = clampT(y, PW ? Ds * qy : Ds);
        const bool ix = cx == x, iy = cy == y;
        if (count && c.owner) cnt += 2 * ((!ix) + (!iy));   // a stored bin stands for k and -k
        if (FULL) mb.template put<2>(u, (uint32_t)ix | ((uint32_t)iy << 1));
        if (rec_f)
          record_f(a, ed_slot0 + u * ed_ustride, (float)(cx - x), (float)(cy - y), t_chk,
                   may_stop && (PW ? fmax(ratioT(fabs(x), qx), ratioT(fabs(y), qy)) : fmax(fabs(x), fabs(y))) <= thr);
        v[u] = mk<T>(cx, cy);
      }
    } else if (clip && FULL) {
      mb.fill();   // nothing clipped
    }
  }
  if (rec && c.live) mb.store(a.mask + (int64_t)t_chk * a.mask_step, mthr);
  if (acc_vb) {
    // persistent callers reduce once per CTA after their last tile
    *acc_vb = max(*acc_vb, mx.dbits(bad));
    *acc_cnt += cnt;
  } else if (!use_mask) {
    unsigned long long vb = mx.dbits(bad), cc = cnt;
    block_max_count(vb, cc, count, s_red);
    if (threadIdx.x == 0) {
      atomicMax(&st.vbits, vb);
      if (cc) atomicAdd(&st.act_f, cc);
    }
  }
  if (a.mode & M_NOWRITE) return;
  fft_pencil<T, L, +1>(v, j, twg, tl);
}

// Check / f-clip pass along the outermost axis (z in 3D, y in 2D): forward
// FFT completes the spectrum; the violation max over all bins is reduced
// (CheckConvergence), Re and Im are clipped to +-D' (ProjectOntoFCube), and
// the inverse FFT of this axis is applied before the store.  Tiles: see
// ChkTile.
template <typename T, int L, int W_ = TileW<T>::value, bool PW = false, int PV = PV_POCS, bool FULL = true, int S = 0>
__device__ __forceinline__ void k_chk_body(const Args& a, const int bx_, const int by_) {
  FFCZ_AXIS_PROLOGUE(T, L, W_, S)
  constexpr int W = G_::W, NT = G_::NT;
  const int M = a.g.M, Nmid = a.g.Nmid;
  const ChkTile c = chk_decode<W>(tile, w, M, Nmid);
  const int64_t estride = (int64_t)Nmid * M;
  const int64_t ustride = (int64_t)NT * estride;
  const v2<T>* in = pick<T>(a, a.sel_in, t_it) + a.g.soff[gi] + c.off + j * estride;
  v2<T> v[V];
#pragma unroll
  for (int u = 0; u < V; ++u) v[u] = in[u * ustride];
  load_tables<T>(s_tw, S ? a.tw1 : a.tw, L, nullptr, nullptr, 0);   // overlaps the loads
  const int nmain = Nmid * (M / W);
  const int ntot = chk_ntiles(W, M, Nmid);
  const int first_tile = bx_ * G_::G;
  const bool cta_has_mirror = first_tile + G_::G - 1 >= nmain && first_tile < ntot;
  const float2* pwb = nullptr;
  int64_t pws = 0;
  if constexpr (PW) pw_pencil(a, gi, c, M, Nmid, estride, pwb, pws);
  chk_core<T, L, TL, PW, PV, FULL>(a, p, st, v, j, w, mthr, c, cta_has_mirror, tl, s_tw, s_red, nullptr, nullptr,
                                   a.g.soff[gi] + c.off + j * estride, ustride, t_it, pwb, pws, 1);
  if ((a.mode & M_NOWRITE) || !c.owner) return;
  v2<T>* out = pick<T>(a, a.sel_out, t_it) + a.g.soff[gi] + c.off + j * estride;
#pragma unroll
  for (int u = 0; u < V; ++u) out[u * ustride] = v[u];
}
template <typename T, int L, int W_ = TileW<T>::value, bool PW = false, int PV = PV_POCS, bool FULL = true, int S = 0>
__global__ void __launch_bounds__(Geo<T, L, W_>::NTHR,
                                  (PW || PV != PV_POCS) ? Geo<T, L, W_>::MINB_PW : Geo<T, L, W_>::MINB)
k_chk(Args a) {
  k_chk_body<T, L, W_, PW, PV, FULL, S>(a, (int)blockIdx.x, (int)blockIdx.y);
}

// ---------------------------------------------------------------------------
// Persistent float32 strided passes fed by TMA
// ---------------------------------------------------------------------------
//
// One CTA per SM slot loops over the tiles of its item; while it transforms
// tile t, the copy engine loads tile t + gridDim.x into the staging buffer,
// so the DRAM latency of a tile hides behind the arithmetic of the previous
// one.  Shared memory: [staging L x W][tile buffer][twiddles][reduction],
// the staging buffer at a 128-byte aligned address.  Tiles of one CTA only
// (G = 1).

template <int L, int W>
struct TmaGeo {
  using G_ = Geo<float, L, W>;
  static_assert(G_::G == 1, "TMA-fed passes use one tile per CTA");
  static constexpr int BOX = L < 256 ? L : 256;        // rows per box
  static constexpr int MINB = 2;                       // CTAs per SM the grid is sized for
  static constexpr size_t stage = (size_t)L * W * sizeof(float2);
  static constexpr size_t bytes =
      128 + stage + (size_t)Tile<float, L, W>::ELEMS * sizeof(float2) + (size_t)L * sizeof(float2) + 32 * 8 * 3 + 32 * 4;
  // the pointwise check pass stages the tile's f-bounds as well
  static constexpr size_t bytes_pw = bytes + stage;
};

#define FFCZ_TMA_PROLOGUE(L_, W_, EXTRA_)                                                \
  using G_ = Geo<float, L_, W_>;                                                         \
  using TL = Tile<float, L_, W_>;                                                        \
  using TG = TmaGeo<L_, W_>;                                                             \
  constexpr int V = G_::V, NT = G_::NT;                                                  \
  extern __shared__ __align__(16) unsigned char smraw[];                                 \
  const uint32_t s0_ = smem_addr(smraw);   /* staging rounded up to 128 bytes below */   \
  float2* s_stage = reinterpret_cast<float2*>(smraw + (((s0_ + 127u) & ~127u) - s0_));  \
  float2* s_tiles = s_stage + L_ * W_ + (EXTRA_); /* EXTRA_: a second staging buffer */ \
  float2* s_tw = s_tiles + TL::ELEMS;                                                    \
  unsigned long long* s_red = reinterpret_cast<unsigned long long*>(s_tw + L_);         \
  __shared__ __align__(8) uint64_t bar;                                                  \
  const int gi = blockIdx.y;                                                             \
  const int item = a.g.item[gi];                                                         \
  const ItemParams& p = a.prm[item];                                                     \
  ItemState& st = a.st[item];                                                            \
  if (!pred_ok(a.pred, st, p)) return;                                                   \
  const int t_it = st.t;                                                                 \
  const int tid = threadIdx.x, w = tid % W_, j = tid / W_;                               \
  const int bin = (a.sel_in == S_CUR) ? (t_it & 1) : ((t_it - 1) & 1);                   \
  if ((smem_addr(s_stage) & 127u) != 0u) {                                               \
    if (tid == 0) atomicExch(a.err, DERR_TMA_ALIGN);                                     \
    return;                                                                              \
  }                                                                                      \
  load_tables<float>(s_tw, a.tw, L_, nullptr, nullptr, 0);                               \
  if (tid == 0) mbar_init(&bar, 1);                                                      \
  __syncthreads();                                                                       \
  uint32_t parity = 0;                                                                   \
  (void)p; (void)NT; (void)s_red;

// Wait for the staging buffer, copy it to registers, release it and start
// the load of the next tile.  After a timeout: DRAIN (waits for the caller's
// other copies in flight), then return (uniformly).
#define FFCZ_TMA_TAKE(ISSUE_NEXT, DRAIN)                                                 \
  {                                                                                      \
    const bool ok_ = mbar_wait_bounded(&bar, parity, kTmaPollLimit);                     \
    if (__syncthreads_or(!ok_)) {                                                        \
      if (tid == 0) atomicExch(a.err, DERR_TMA_TIMEOUT);                                 \
      mbar_wait_bounded(&bar, parity, kTmaPollLimit); /* copies still in flight */       \
      DRAIN;                                                                             \
      return;                                                                            \
    }                                                                                    \
    _Pragma("unroll") for (int u = 0; u < V; ++u) v[u] = s_stage[(j + u * NT) * W + w]; \
    __syncthreads();                                                                     \
    if (tid == 0) { ISSUE_NEXT; }                                                        \
    parity ^= 1u;                                                                        \
  }

template <int L, int DIR, int W>
__global__ void __launch_bounds__(Geo<float, L, W>::NTHR, TmaGeo<L, W>::MINB)
k_axis_tma(Args a) {
  FFCZ_TMA_PROLOGUE(L, W, 0)
  const int M = a.g.M;
  const int tpr = M / W;
  const int ntiles = a.g.Nz * tpr;
  const CUtensorMap* map = a.tm_axis + 2 * gi + bin;
  // tile t: pencils kx0..kx0+W-1 of plane z; rows z L + y of the [Nz L][M] view
  auto issue = [&](int t) {
    const int x = (t % tpr) * W, y0 = (t / tpr) * L;
    mbar_arrive_expect_tx(&bar, (uint32_t)TG::stage);
#pragma unroll
    for (int b = 0; b < L / TG::BOX; ++b) tma_load_2d(s_stage + b * TG::BOX * W, map, x, y0 + b * TG::BOX, &bar);
  };
  int tile = blockIdx.x;
  if (tid == 0 && tile < ntiles) issue(tile);
  float2* outb = pick<float>(a, a.sel_out, t_it) + a.g.soff[gi];
  while (tile < ntiles) {
    const int next = tile + gridDim.x;
    float2 v[V];
    FFCZ_TMA_TAKE(if (next < ntiles) { fence_proxy_async_smem(); issue(next); }, (void)0)
    TL tl{s_tiles + w, false};
    fft_pencil<float, L, DIR>(v, j, s_tw, tl);
    const int z = tile / tpr, kx = (tile % tpr) * W + w;
    float2* out = outb + (int64_t)z * L * M + kx + (int64_t)j * M;
#pragma unroll
    for (int u = 0; u < V; ++u) out[(int64_t)u * NT * M] = v[u];
    __syncthreads();   // the tile buffer is reused by the next tile
    tile = next;
  }
}

// Pointwise bounds staged in shared memory by the copy engine: chk_core
// waits (bounded) for the tile's load after its forward transform; a
// timeout raises *late_flag, on which the caller stops.
struct QStaged {
  static constexpr bool late = true;
  uint32_t sq;      // shared-memory address of the staged bounds of pencil w
  uint64_t* b;
  uint32_t par;
  bool on;
  bool* late_flag;
  __device__ __forceinline__ void operator()() const {
    if (on && !mbar_wait_bounded(b, par, kTmaPollLimit)) *late_flag = true;
  }
};

// AUX: the pass stages an auxiliary packed field per main tile beside the
// spectrum: the pointwise f-bounds (PW) or the Dykstra / Douglas-Rachford
// residual (read before this pass rewrites it in place).
template <int L, int W, bool FULL = true, bool PW = false, int PV = PV_POCS>
__global__ void __launch_bounds__(Geo<float, L, W>::NTHR, TmaGeo<L, W>::MINB)
k_chk_tma(Args a) {
  constexpr bool AUX = PW || PV == PV_DYKSTRA || PV == PV_DR;
  FFCZ_TMA_PROLOGUE(L, W, AUX ? L * W : 0)
  const int M = a.g.M, Nmid = a.g.Nmid;
  const int tpr = M / W;
  const int nmain = Nmid * tpr;
  const int ntot = chk_ntiles(W, M, Nmid);
  const int64_t estride = (int64_t)Nmid * M;
  const CUtensorMap* map = a.tm_chk + 2 * gi + bin;
  // main tile t: pencils kx0..kx0+W-1 at middle index mid; [Nz][Nmid M] view
  auto issue = [&](int t) {
    const int x = (t / tpr) * M + (t % tpr) * W;
    mbar_arrive_expect_tx(&bar, (uint32_t)TG::stage);
#pragma unroll
    for (int b = 0; b < L / TG::BOX; ++b) tma_load_2d(s_stage + b * TG::BOX * W, map, x, b * TG::BOX, &bar);
  };
  // the auxiliary field of a main tile goes to its own staging buffer (same
  // view), loaded once the previous tile has used its copy, and waited for
  // after the forward transform
  float2* s_pw = s_stage + L * W;
  __shared__ __align__(8) uint64_t bar_pw;
  uint32_t par_pw = 0;
  bool pw_late = false;   // a wait for the staged bounds ran out
  auto issue_pw = [&](int t) {
    const int x = (t / tpr) * M + (t % tpr) * W;
    mbar_arrive_expect_tx(&bar_pw, (uint32_t)TG::stage);
#pragma unroll
    for (int b = 0; b < L / TG::BOX; ++b) tma_load_2d(s_pw + b * TG::BOX * W, a.tm_aux + gi, x, b * TG::BOX, &bar_pw);
  };
  if constexpr (AUX) {
    if (tid == 0) mbar_init(&bar_pw, 1);
    __syncthreads();
  }
  int tile = blockIdx.x;
  if (tid == 0 && tile < nmain) {
    issue(tile);
    if constexpr (AUX) issue_pw(tile);
  }
  const float2* inb = pick<float>(a, a.sel_in, t_it) + a.g.soff[gi];
  float2* outb = pick<float>(a, a.sel_out, t_it) + a.g.soff[gi];
  unsigned long long acc_vb = 0ull, acc_cnt = 0ull;
  while (tile < ntot) {
    const int next = tile + gridDim.x;
    const ChkTile c = chk_decode<W>(tile, w, M, Nmid);
    float2 v[V];
    if (tile < nmain) {
      FFCZ_TMA_TAKE(if (next < nmain) { fence_proxy_async_smem(); issue(next); },
                    if (AUX) mbar_wait_bounded(&bar_pw, par_pw, kTmaPollLimit))
    } else {
      // kx = 0 mirror pencils are not one box: plain loads
      const float2* in = inb + c.off + j * estride;
#pragma unroll
      for (int u = 0; u < V; ++u) v[u] = in[(int64_t)u * NT * estride];
    }
    TL tl{s_tiles + w, false};
    const int64_t mthr = (int64_t)gi * a.mask_thr + (int64_t)tile * G_::TPT + tid;
    const float2* pwb = nullptr;
    int64_t pws = 0;
    const bool main_tile = tile < nmain;
    if constexpr (PW) {
      if (main_tile) { pwb = s_pw + w; pws = W; }
      else pw_pencil(a, gi, c, M, Nmid, estride, pwb, pws);
    }
    using QW = typename std::conditional<AUX, QStaged, QEarly>::type;
    QW qw{};
    if constexpr (AUX) qw = QStaged{smem_addr(s_pw + w), &bar_pw, par_pw, main_tile, &pw_late};
    chk_core<float, L, TL, PW, PV, FULL, QW>(a, p, st, v, j, w, mthr, c, tile >= nmain, tl, s_tw, s_red,
                                                  &acc_vb, &acc_cnt, a.g.soff[gi] + c.off + j * estride,
                                                  (int64_t)NT * estride, t_it, pwb, pws, 1, qw);
    if (!(a.mode & M_NOWRITE) && c.owner) {
      float2* out = outb + c.off + j * estride;
#pragma unroll
      for (int u = 0; u < V; ++u) out[(int64_t)u * NT * estride] = v[u];
    }
    if constexpr (AUX) {
      // the tile buffer and the auxiliary staging are reused by the next tile
      if (__syncthreads_or(pw_late)) {
        if (tid == 0) atomicExch(a.err, DERR_TMA_TIMEOUT);
        mbar_wait_bounded(&bar_pw, par_pw, kTmaPollLimit);                   // copies still in flight
        if (main_tile && next < nmain) mbar_wait_bounded(&bar, parity, kTmaPollLimit);
        return;
      }
      if (main_tile) {
        par_pw ^= 1u;
        if (tid == 0 && next < nmain) { fence_proxy_async_smem(); issue_pw(next); }
      }
    } else {
      __syncthreads();   // the tile buffer is reused by the next tile
    }
    tile = next;
  }
  if (!(a.mode & M_MASK)) {
    block_max_count(acc_vb, acc_cnt, (a.mode & M_COUNT) != 0, s_red);
    if (threadIdx.x == 0) {
      atomicMax(&st.vbits, acc_vb);
      if (acc_cnt) atomicAdd(&st.act_f, acc_cnt);
    }
  }
}

// Persistent float32 x pass (C2R, s-clip, R2C) fed by bulk copies (ED: the
// full form with edit recording and the adjoint modes, else lean): a CTA
// holds G tiles of W rows each (one warp per tile); its G W consecutive rows
// are one contiguous block of the packed spectrum, loaded by a single
// cp.async.bulk while the previous block is transformed.  Shared memory:
// [staging G W M][G tile buffers][twiddles][R2C twiddles][reduction].
// The staged rows are RS = M + PAD values apart: the PAD (16 / W values, an
// even count, so every row starts on a 16-byte boundary) puts the W rows a
// half-warp reads at once in different banks.
template <int M, int W>
struct PxTmaGeo {
  using G_ = Geo<float, M, W>;
  static constexpr int RG = G_::G * W;                     // rows per block
  static constexpr int PAD = (W >= 2 && W <= 8) ? 16 / W : 0;
  static constexpr int RS = M + PAD;                       // staged row stride
  static constexpr size_t stage = (size_t)RG * RS * sizeof(float2);
  static constexpr size_t bytes = 128 + stage + (size_t)G_::G * Tile<float, M, W>::ELEMS * sizeof(float2) +
                                  2 * (size_t)M * sizeof(float2) + 32 * 8 * 3 + 32 * 4;
};

// One block of rows r0 .. r0 + RG - 1 (fewer at the end) into the staging
// buffer at row stride RS: one bulk copy per row when the rows are padded.
template <int M, int W>
__device__ __forceinline__ void px_stage_rows(float2* s_stage, const float2* inb, int64_t r0, int64_t rows,
                                              uint64_t* bar) {
  using PG = PxTmaGeo<M, W>;
  const int64_t nr = rows - r0 < PG::RG ? rows - r0 : PG::RG;
  const uint32_t rb = (uint32_t)(M * sizeof(float2));
  mbar_arrive_expect_tx(bar, (uint32_t)nr * rb);
  if constexpr (PG::PAD == 0) {
    bulk_load(s_stage, inb + r0 * M, (uint32_t)nr * rb, bar);
  } else {
    for (int r = 0; r < (int)nr; ++r) bulk_load(s_stage + r * PG::RS, inb + (r0 + r) * M, rb, bar);
  }
}

template <int M, int W, bool ED = false, bool PW = false, int PV = PV_POCS>
__global__ void __launch_bounds__(Geo<float, M, W>::NTHR,
                                  (PW || PV != PV_POCS) ? Geo<float, M, W>::MINB_PW : Geo<float, M, W>::MINB)
k_px_tma(Args a) {
  using G_ = Geo<float, M, W>;
  using TL = Tile<float, M, W>;
  using PG = PxTmaGeo<M, W>;
  constexpr int V = G_::V, NT = G_::NT, RG = PG::RG;
  extern __shared__ __align__(16) unsigned char smraw[];
  const uint32_t s0 = smem_addr(smraw);   // staging rounded up to 128 bytes
  float2* s_stage = reinterpret_cast<float2*>(smraw + (((s0 + 127u) & ~127u) - s0));
  float2* s_tiles = s_stage + RG * PG::RS;
  float2* s_tw = s_tiles + G_::G * TL::ELEMS;
  float2* s_twr = s_tw + M;
  unsigned long long* s_red = reinterpret_cast<unsigned long long*>(s_twr + M);
  __shared__ __align__(8) uint64_t bar;
  const int gi = blockIdx.y;
  const int item = a.g.item[gi];
  const ItemParams& p = a.prm[item];
  ItemState& st = a.st[item];
  if (!pred_ok(a.pred, st, p)) return;
  const int t_it = st.t;
  const int g = threadIdx.x / G_::TPT, tid = threadIdx.x % G_::TPT;
  const int w = tid % W, j = tid / W;
  const int64_t rows = a.g.rows;
  const int64_t nblk = (rows + RG - 1) / RG;
  const float2* inb = pick<float>(a, a.sel_in, t_it) + a.g.soff[gi];
  float2* outb = pick<float>(a, a.sel_out, t_it) + a.g.soff[gi];
  if ((smem_addr(s_stage) & 127u) != 0u || (reinterpret_cast<uintptr_t>(inb) & 15u) != 0u) {
    if (threadIdx.x == 0) atomicExch(a.err, DERR_TMA_ALIGN);
    return;
  }
  load_tables<float>(s_tw, a.tw, M, s_twr, a.twr, M);
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t parity = 0;
  auto issue = [&](int64_t blk) { px_stage_rows<M, W>(s_stage, inb, blk * RG, rows, &bar); };
  int64_t blk = blockIdx.x;
  if (threadIdx.x == 0 && blk < nblk) issue(blk);
  unsigned long long cnt = 0;
  AbsMax<float> svm;   // ADMM: max |a_t| over the CTA's points
  while (blk < nblk) {
    const int64_t next = blk + gridDim.x;
    const bool ok = mbar_wait_bounded(&bar, parity, kTmaPollLimit);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(a.err, DERR_TMA_TIMEOUT);
      mbar_wait_bounded(&bar, parity, kTmaPollLimit);   // copies still in flight
      return;
    }
    float2 v[V];
#pragma unroll
    for (int u = 0; u < V; ++u) v[u] = s_stage[(g * W + w) * PG::RS + j + u * NT];
    __syncthreads();
    if (threadIdx.x == 0 && next < nblk) {
      fence_proxy_async_smem();
      issue(next);
    }
    parity ^= 1u;
    const int tile = (int)(blk * G_::G + g);
    const int64_t prow = (int64_t)tile * W + w;
    const bool live = prow < rows;
    const int64_t row = live ? prow : 0;
    const int64_t mthr = (int64_t)gi * a.mask_thr + (int64_t)tile * G_::TPT + tid;
    TL tl{s_tiles + g * TL::ELEMS + w, false};
    float2* edrow = a.ed_s ? reinterpret_cast<float2*>(a.ed_s + a.g.eoff[gi]) + row * M : nullptr;
    const float2* ebrow = PW ? reinterpret_cast<const float2*>(a.pw_e + a.g.eoff[gi]) + row * M : nullptr;
    const float2* qin = nullptr;
    float2* qout = nullptr;
    if constexpr (PV != PV_POCS) {   // Dykstra's q / ADMM's u, one buffer per iteration parity
      qin = reinterpret_cast<const float2*>(a.pv_q[(t_it - 1) & 1] + a.g.eoff[gi]) + row * M;
      qout = reinterpret_cast<float2*>(a.pv_q[t_it & 1] + a.g.eoff[gi]) + row * M;
    }
    cnt += px_core<float, M, TL, PW, ED, PV>(a, p, v, j, mthr, row, live, t_it, a.g.eoff[gi], tl, s_tw, s_twr,
                                             edrow, ebrow, qin, qout, &svm);
    if (live) {
      float2* out = outb + row * M;
#pragma unroll
      for (int u = 0; u < V; ++u) out[j + u * NT] = v[u];
    }
    TL::sync();   // the warp's tile buffer is reused by the next block
    blk = next;
  }
  if constexpr (PV == PV_ADMM) {
    // spatial check of a_t over the CTA's rows (NaN -> +inf)
    unsigned long long vb = svm.dbits(svm.val() != svm.val()), cz = 0ull;
    block_max_count(vb, cz, false, s_red);
    if (threadIdx.x == 0) atomicMax(&st.svbits, vb);
  }
  if (a.mode & M_COUNT) {
    Red r{0ull, 0.0, cnt};
    block_reduce(r, s_red);
    if (threadIdx.x == 0 && r.cnt) atomicAdd(&st.act_s, r.cnt);
  }
}

// After a loop: a marginal frequency edit recorded at the check that
// stopped the loop (index T = the item's iteration count; Alg. 1 projects
// nothing there) is taken back; the other marks are cleared.  Every slot of
// every member of the group; grid (x: slots, y: members).
static __global__ void k_edits_finalize(Group g, const ItemState* st, float2* ed_f, float2* ed_p,
                                        int* ed_t, int64_t slots_per_item) {
  const int gi = blockIdx.y;
  const int T = st[g.item[gi]].t;
  const int64_t base = g.soff[gi];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < slots_per_item;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int tg = ed_t[base + i];
    if (tg == 0) continue;
    if (tg - 1 == T) {
      float2 f = ed_f[base + i];
      const float2 q = ed_p[base + i];
      f.x -= q.x;
      f.y -= q.y;
      ed_f[base + i] = f;
    }
    ed_t[base + i] = 0;
    ed_p[base + i] = make_float2(0.f, 0.f);
  }
}

// The same for 1D items, whose frequency edits are kept on their half
// spectrum (bins k <= N/2 at the item's canonical offset).
static __global__ void k_edits_finalize1(Group g, const ItemParams* prm, const ItemState* st, float2* ed_f,
                                         float2* ed_p, int* ed_t) {
  const int gi = blockIdx.y;
  const int item = g.item[gi];
  const int T = st[item].t;
  const int64_t base = g.coff[gi], slots = prm[item].n / 2 + 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < slots;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int tg = ed_t[base + i];
    if (tg == 0) continue;
    if (tg - 1 == T) {
      float2 f = ed_f[base + i];
      const float2 q = ed_p[base + i];
      f.x -= q.x;
      f.y -= q.y;
      ed_f[base + i] = f;
    }
    ed_t[base + i] = 0;
    ed_p[base + i] = make_float2(0.f, 0.f);
  }
}

// Pointwise bounds of every member of a group: counts non-positive or
// non-finite bounds into *bad and takes min_k Delta_k (Re and Im) per item
// into minbits (positive floats order like their bit patterns).  Grid
// (x: any, y: members).
static __global__ void k_pw_check(Group g, const float* pw_e, const float2* pw_f, int64_t npt, int64_t nb,
                                  unsigned int* minbits, int* bad) {
  const int gi = blockIdx.y;
  const int item = g.item[gi];
  const float* eb = pw_e + g.eoff[gi];
  const float2* fb = pw_f + g.coff[gi];
  int nbad = 0;
  float mn = INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npt; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = eb[i];
    nbad += !(v >= FLT_MIN && v <= FLT_MAX);   // normal, finite, positive
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 q = fb[i];
    nbad += !(q.x >= FLT_MIN && q.x <= FLT_MAX) + !(q.y >= FLT_MIN && q.y <= FLT_MAX);
    mn = fminf(mn, fminf(q.x, q.y));
  }
  for (int o = 16; o > 0; o >>= 1) {
    nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (nbad) atomicAdd(bad, nbad);
    if (mn > 0.f) atomicMin(minbits + item, __float_as_uint(mn));
  }
}
// The same for 1D items, whose members differ in length: N spatial bounds
// and N/2 + 1 (Delta^Re, Delta^Im) pairs (bins k <= N/2; bin N - k uses
// those of k) per member.
static __global__ void k_pw_check1(Group g, const ItemParams* prm, const float* pw_e, const float2* pw_f,
                                   unsigned int* minbits, int* bad) {
  const int gi = blockIdx.y;
  const int item = g.item[gi];
  const int64_t npt = prm[item].n, nb = npt / 2 + 1;
  const float* eb = pw_e + g.eoff[gi];
  const float2* fb = pw_f + g.coff[gi];
  int nbad = 0;
  float mn = INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npt; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = eb[i];
    nbad += !(v >= FLT_MIN && v <= FLT_MAX);
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 q = fb[i];
    nbad += !(q.x >= FLT_MIN && q.x <= FLT_MAX) + !(q.y >= FLT_MIN && q.y <= FLT_MAX);
    mn = fminf(mn, fminf(q.x, q.y));
  }
  for (int o = 16; o > 0; o >>= 1) {
    nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (nbad) atomicAdd(bad, nbad);
    if (mn > 0.f) atomicMin(minbits + item, __float_as_uint(mn));
  }
}

// The caller's (Delta^Re, Delta^Im) on the canonical half spectrum
// [Nz][Nmid][M+1] into the check pass's layouts: the packed slots kx of each
// row (1 <= kx < M; slot 0 also gets the kx = 0 bounds) and one float4 per
// row for the kx = 0 (A) and kx = Nx/2 (B) planes.
static __global__ void k_pw_pack(Group g, const float2* canon, float2* packed, float2* mirror2, int64_t nb) {
  const int gi = blockIdx.y;
  const int M = g.M;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / (M + 1);
    const int kx = (int)(i - row * (M + 1));
    const float2 b = canon[g.coff[gi] + i];
    if (kx < M) packed[g.soff[gi] + row * M + kx] = b;
    if (kx == 0) mirror2[2 * (g.roff[gi] + row)] = b;
    if (kx == M) mirror2[2 * (g.roff[gi] + row) + 1] = b;
  }
}

static __global__ void k_pw_scale(ItemParams* prm, const unsigned int* minbits, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) prm[i].bscale = 1.0 / (double)__uint_as_float(minbits[i]);
}

// ---------------------------------------------------------------------------
// Per-item control kernels
// ---------------------------------------------------------------------------

// Loop decision after a check (Alg. 1: break when CheckConvergence passes;
// readings: stop at v <= D(1 - eta/2) once t >= min_iters, cap at max_iters).
// Persistent float32 entry x pass (e rows -> packed spectrum, with the
// max |e|, sum e^2 and NaN measurement) fed by bulk copies of blocks of rows,
// the same way as k_px_tma (no pre-clip, mask or pointwise bounds: those use
// k_xfwd).  Each thread sums its squares per block in float32 (at most 2V
// terms, inflated as in k_xfwd) and the blocks in double.
template <int M, int W, bool PW = false>
__global__ void __launch_bounds__(Geo<float, M, W>::NTHR, Geo<float, M, W>::MINB)
k_xfwd_tma(Args a) {
  using G_ = Geo<float, M, W>;
  using TL = Tile<float, M, W>;
  using PG = PxTmaGeo<M, W>;
  constexpr int V = G_::V, NT = G_::NT, RG = PG::RG;
  extern __shared__ __align__(16) unsigned char smraw[];
  const uint32_t s0 = smem_addr(smraw);   // staging rounded up to 128 bytes
  float2* s_stage = reinterpret_cast<float2*>(smraw + (((s0 + 127u) & ~127u) - s0));
  float2* s_tiles = s_stage + RG * PG::RS;
  float2* s_tw = s_tiles + G_::G * TL::ELEMS;
  float2* s_twr = s_tw + M;
  unsigned long long* s_red = reinterpret_cast<unsigned long long*>(s_twr + M);
  __shared__ __align__(8) uint64_t bar;
  const int gi = blockIdx.y;
  const int item = a.g.item[gi];
  const ItemParams& p = a.prm[item];
  ItemState& st = a.st[item];
  if (!pred_ok(a.pred, st, p)) return;
  const int t_it = st.t;
  const int g = threadIdx.x / G_::TPT, tid = threadIdx.x % G_::TPT;
  const int w = tid % W, j = tid / W;
  const int64_t rows = a.g.rows;
  const int64_t nblk = (rows + RG - 1) / RG;
  const float2* inb = reinterpret_cast<const float2*>(a.e + a.g.eoff[gi]);
  float2* outb = pick<float>(a, a.sel_out, t_it) + a.g.soff[gi];
  if ((smem_addr(s_stage) & 127u) != 0u || (reinterpret_cast<uintptr_t>(inb) & 15u) != 0u) {
    if (threadIdx.x == 0) atomicExch(a.err, DERR_TMA_ALIGN);
    return;
  }
  load_tables<float>(s_tw, a.tw, M, s_twr, a.twr, M);
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t parity = 0;
  auto issue = [&](int64_t blk) { px_stage_rows<M, W>(s_stage, inb, blk * RG, rows, &bar); };
  int64_t blk = blockIdx.x;
  if (threadIdx.x == 0 && blk < nblk) issue(blk);
  const bool measure = (a.mode & M_MEASURE) != 0;
  AbsMax<float> mx;
  bool bad = false;
  double ssq_d = 0.0;
  while (blk < nblk) {
    const int64_t next = blk + gridDim.x;
    const bool ok = mbar_wait_bounded(&bar, parity, kTmaPollLimit);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(a.err, DERR_TMA_TIMEOUT);
      mbar_wait_bounded(&bar, parity, kTmaPollLimit);   // copies still in flight
      return;
    }
    const int tile = (int)(blk * G_::G + g);
    const int64_t prow = (int64_t)tile * W + w;
    const bool live = prow < rows;
    const int64_t row = live ? prow : 0;
    float2 v[V];
    float ssq = 0.f;
    const float2* ebrow = PW ? reinterpret_cast<const float2*>(a.pw_e + a.g.eoff[gi]) + row * M : nullptr;
#pragma unroll
    for (int u = 0; u < V; ++u) {
      v[u] = s_stage[(g * W + w) * PG::RS + j + u * NT];
      if (measure && live) {
        if constexpr (PW) {   // pointwise E_n: the maximum of |e_n| / E_n
          const float2 eb = ebrow[j + u * NT];
          mx.add(ratioT(v[u].x, eb.x)); mx.add(ratioT(v[u].y, eb.y));
        } else {
          mx.add(v[u].x); mx.add(v[u].y);
        }
        bad |= (v[u].x != v[u].x) | (v[u].y != v[u].y);
        ssq = fmaf(v[u].x, v[u].x, fmaf(v[u].y, v[u].y, ssq));
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && next < nblk) {
      fence_proxy_async_smem();
      issue(next);
    }
    parity ^= 1u;
    ssq_d += (double)ssq * (1.0 + 0x1p-17);   // 2V float32 terms: relative error < (2V+1) u32
    TL tl{s_tiles + g * TL::ELEMS + w, false};
    fft_pencil<float, M, -1>(v, j, s_tw, tl);
    r2c_post<float, M>(v, j, tl, s_twr);
    if (live) {
      float2* out = outb + row * M;
#pragma unroll
      for (int u = 0; u < V; ++u) out[j + u * NT] = v[u];
    }
    TL::sync();   // the warp's tile buffer is reused by the next block
    blk = next;
  }
  if (measure) {
    Red r{mx.dbits(bad), ssq_d, 0ull};
    block_reduce(r, s_red);
    if (threadIdx.x == 0) {
      atomicMax(&st.emaxbits, r.vbits);
      atomicAdd(&st.sumsq, r.sum);
    }
  }
}

// Persistent float32 exit x pass (C2R, scale 1/N, s-clip, store or add to
// e) fed by bulk copies of blocks of spectrum rows, the same way as
// k_px_tma; Alg. 1 and pointwise bounds (the Dykstra exit uses k_xexit).
template <int M, int W, bool PW = false>
__global__ void __launch_bounds__(Geo<float, M, W>::NTHR, PW ? Geo<float, M, W>::MINB_PW : Geo<float, M, W>::MINB)
k_xexit_tma(Args a) {
  using G_ = Geo<float, M, W>;
  using TL = Tile<float, M, W>;
  using PG = PxTmaGeo<M, W>;
  constexpr int V = G_::V, NT = G_::NT, RG = PG::RG;
  extern __shared__ __align__(16) unsigned char smraw[];
  const uint32_t s0 = smem_addr(smraw);   // staging rounded up to 128 bytes
  float2* s_stage = reinterpret_cast<float2*>(smraw + (((s0 + 127u) & ~127u) - s0));
  float2* s_tiles = s_stage + RG * PG::RS;
  float2* s_tw = s_tiles + G_::G * TL::ELEMS;
  float2* s_twr = s_tw + M;
  __shared__ __align__(8) uint64_t bar;
  const int gi = blockIdx.y;
  const int item = a.g.item[gi];
  const ItemParams& p = a.prm[item];
  ItemState& st = a.st[item];
  if (!pred_ok(a.pred, st, p)) return;
  const int t_it = st.t;
  const int g = threadIdx.x / G_::TPT, tid = threadIdx.x % G_::TPT;
  const int w = tid % W, j = tid / W;
  const int64_t rows = a.g.rows;
  const int64_t nblk = (rows + RG - 1) / RG;
  const float2* inb = pick<float>(a, a.sel_in, t_it) + a.g.soff[gi];
  if ((smem_addr(s_stage) & 127u) != 0u || (reinterpret_cast<uintptr_t>(inb) & 15u) != 0u) {
    if (threadIdx.x == 0) atomicExch(a.err, DERR_TMA_ALIGN);
    return;
  }
  load_tables<float>(s_tw, a.tw, M, s_twr, a.twr, M);
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t parity = 0;
  auto issue = [&](int64_t blk) { px_stage_rows<M, W>(s_stage, inb, blk * RG, rows, &bar); };
  int64_t blk = blockIdx.x;
  if (threadIdx.x == 0 && blk < nblk) issue(blk);
  while (blk < nblk) {
    const int64_t next = blk + gridDim.x;
    const bool ok = mbar_wait_bounded(&bar, parity, kTmaPollLimit);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(a.err, DERR_TMA_TIMEOUT);
      mbar_wait_bounded(&bar, parity, kTmaPollLimit);   // copies still in flight
      return;
    }
    float2 v[V];
#pragma unroll
    for (int u = 0; u < V; ++u) v[u] = s_stage[(g * W + w) * PG::RS + j + u * NT];
    __syncthreads();
    if (threadIdx.x == 0 && next < nblk) {
      fence_proxy_async_smem();
      issue(next);
    }
    parity ^= 1u;
    const int tile = (int)(blk * G_::G + g);
    const int64_t prow = (int64_t)tile * W + w;
    const bool live = prow < rows;
    const int64_t row = live ? prow : 0;
    TL tl{s_tiles + g * TL::ELEMS + w, false};
    // pointwise E_n of the thread's points, loaded before the transform
    const float2* ebrow = PW ? reinterpret_cast<const float2*>(a.pw_e + a.g.eoff[gi]) + row * M : nullptr;
    float2 ebr[PW ? V : 1];
    if constexpr (PW) {
#pragma unroll
      for (int u = 0; u < V; ++u) ebr[u] = ebrow[j + u * NT];
    }
    c2r_pre<float, M>(v, j, tl, s_twr);
    fft_pencil<float, M, +1>(v, j, s_tw, tl);
    float2* erow = reinterpret_cast<float2*>(a.e + a.g.eoff[gi]) + row * M;
    if (live) xexit_store<float, V, PW, PV_POCS>(a, p, v, j, NT, erow, ebrow, nullptr, PW ? ebr : nullptr);
    TL::sync();   // the warp's tile buffer is reused by the next block
    blk = next;
  }
}

// s_check: ADMM loops, whose candidate after iteration t >= 1 is a_t (inside
// F' by construction) and whose stopping test is max|a_t| <= E(1 - eta/2).
static __global__ void k_decide(const ItemParams* prm, ItemState* st, int n, int* n_active, int s_check = 0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ItemState& s = st[i];
  if (s.done) return;
  const ItemParams& p = prm[i];
  double v = __longlong_as_double((long long)s.vbits);
  double thr = p.thr;
  s.vbits = 0ull;
  s.f_ratio = v / p.D;
  if (s_check && s.t >= 1) {
    const double sv = __longlong_as_double((long long)s.svbits);
    if (!(sv <= DBL_MAX)) v = sv;   // non-finite either way
    else if (v <= DBL_MAX) { v = sv; thr = p.thrs; s.f_ratio = sv / p.E; }
  }
  s.svbits = 0ull;
  s.last_act_s = s.act_s;
  s.last_act_f = s.prev_act_f;
  s.prev_act_f = s.act_f;
  s.act_s = 0ull;
  s.act_f = 0ull;
  int done = 0;
  if (!(v <= DBL_MAX)) { done = 1; s.status = 6; }
  else if (v <= thr && s.t >= p.min_iters) { done = 1; s.status = 0; }
  else if (s.t >= p.max_iters) { done = 1; s.status = 4; }
  if (done) {
    s.done = 1;
    atomicSub(n_active, 1);
  } else {
    s.t += 1;
  }
}

// Initialise loop state; items with pred P_UNCERT set only reset those not
// yet certified (repair rounds).
static __global__ void k_init(ItemState* st, int n, int only_uncertified, int* n_active) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ItemState& s = st[i];
  const bool run = !only_uncertified || !s.certified;
  s.vbits = 0ull; s.svbits = 0ull; s.emaxbits = 0ull; s.sumsq = 0.0;
  s.act_s = s.act_f = 0ull; s.last_act_s = s.last_act_f = s.prev_act_f = 0ull;
  s.t = 0;
  s.done = run ? 0 : 1;
  if (!only_uncertified) { s.status = 0; s.preclip = 0; s.certified = 0; s.repairs = 0; s.f_ratio = 0.0; }
  if (run) atomicAdd(n_active, 1);
}

static __global__ void k_mark_preclip(const ItemParams* prm, ItemState* st, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double emax = __longlong_as_double((long long)st[i].emaxbits);
  if (emax > prm[i].E) st[i].preclip = 1;
  if (!(emax <= DBL_MAX)) st[i].preclip = 0;
}

// Certification: max|e| <= E and violation + b <= D, with b a bound on the
// FP64 FFT's rounding error: |err_k| <= ||err||_2 <= c (log2 N + 2) u ||y||_2,
// ||y||_2 = sqrt(N sum e^2) (Parseval), u = 2^-53, c = 10 (>= the per-level
// constant of radix-2 butterflies with rounded twiddles, radix 4/8 being
// compositions of them).
// vscale: the factor that undoes an exact power-of-two scaling of the
// certification transform (0.5 when its x pass returned 2 X).
static __global__ void k_certify(const ItemParams* prm, ItemState* st, int n, int repair_round,
                                 double vscale = 1.0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ItemState& s = st[i];
  const ItemParams& p = prm[i];
  if (repair_round && s.certified) return;
  const double emax = __longlong_as_double((long long)s.emaxbits);
  const double v = vscale * __longlong_as_double((long long)s.vbits);
  const double ln = log2((double)p.n);
  // ||e||_2 from above, two ways: the float32 partial sums of squares (each
  // inflated for its rounding) plus at most 2^-126 per point for squares
  // that fell below the float32 normal range, and sqrt(N) max|e| (exact);
  // the first overflows for |e| beyond about 2^63, the second is looser
  // when a few points dominate, so the smaller one is used
  // (with pointwise bounds emax is max |e_n| / E_n, not a bound on |e_n|:
  // only the sum of squares of the values bounds the norm there)
  const double ssq = s.sumsq + (double)p.n * 0x1p-126;
  const double nrm_max = sqrt((double)p.n) * emax;
  const double nrm = p.pw ? sqrt(ssq) : (ssq <= DBL_MAX) ? fmin(sqrt(ssq), nrm_max) : nrm_max;
  double b = 10.0 * (ln + 2.0) * 1.1102230246251565e-16 * sqrt((double)p.n) * nrm;
  if (p.logP > 0) {
    // Bluestein: FFT_P, product with Bt (|Bt_k| <= 2N), IFFT_P and two chirp
    // products; |err_k| <= ||err||_2 <= c (2 log2 P + 6) u 2N ||x||_2
    b = 10.0 * (2.0 * p.logP + 6.0) * 1.1102230246251565e-16 * 2.0 * (double)p.n * nrm;
    if (p.h1) {
      // through Z = DFT_{N/2}(x_2n + i x_2n+1) (length P/2, ||z||_2 = ||x||_2):
      // |dZ| <= b_Z = c (2 log2 (P/2) + 6) u N ||x||_2; X_k = (A - i W B)/2 is
      // linear in Z_k, conj Z_{N/2-k} with coefficients of modulus <= 1, so the
      // error of Z adds at most 2 b_Z, and the rounding of A, B, W B (W within
      // a few ulps) and the sum at most 10 u (|Z_k| + |Z_{N/2-k}|) <= 20 u sqrt(N) ||x||_2
      const double bz = 10.0 * (2.0 * (p.logP - 1) + 6.0) * 1.1102230246251565e-16 * (double)p.n * nrm;
      b = 2.0 * bz + 20.0 * 1.1102230246251565e-16 * sqrt((double)p.n) * nrm;
    }
  }
  s.v64 = v;
  s.emax64 = emax;
  s.bound64 = b * p.bscale;   // in the units of v (pointwise: relative to min Delta_k)
  s.certified = (emax <= p.E) && (v + s.bound64 <= p.D);
  s.vbits = 0ull;
  s.emaxbits = 0ull;
  s.sumsq = 0.0;
}

// g <- g * [|e0| <= E'] for items whose input was pre-clipped (adjoint of
// the pre-loop s-projection).
static __global__ void k_premask(float* g, const float* e0, const ItemParams* prm, const ItemState* st,
                          int item, int64_t n) {
  if (!st[item].preclip) return;
  const float Es = prm[item].Esf;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float x = e0[i];
    if (!(fabsf(x) <= Es)) g[i] = 0.f;
  }
}

}  // namespace ffcz
