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

#include "fft_core.cuh"

namespace ffcz {

struct ItemParams {
  double E, D, Es, Ds, thr, inv_n;   // bounds, shrunk bounds, stop threshold, 1/N
  float Esf, Dsf, thrf, inv_nf;      // the same in float32
  int64_t n;                         // points
  int32_t min_iters, max_iters;
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
};

struct Group {
  int32_t ndim, Nz, Nmid, M;     // chk-axis length, middle-axis length (1 in 2D), Nx/2
  int64_t rows;                  // x-rows per item (N / Nx)
  const int32_t* item;           // global item index of each group member
  const int64_t* eoff;           // float offset of each member in e
  const int64_t* soff;           // complex offset of each member's spectrum
};

enum Pred : int { P_ALL = 0, P_ACTIVE = 1, P_EXIT = 2, P_PRECLIP = 3, P_UNCERT = 4 };
enum Sel : int { S_CUR = 0, S_PREV = 1 };
enum Mode : int {
  M_CLIP = 1, M_MASK = 2, M_RECORD = 4, M_MEASURE = 8, M_PRECLIP = 16, M_NOWRITE = 32,
  M_CKPT = 64
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
  float* ckpt;             // checkpoint buffer for e_t
  int ckpt_every;
  int pred, sel_in, sel_out, mode;
  const void* tw;          // exp(-2 pi i m / L), m < L
  const void* twr;         // exp(-2 pi i k / Nx), k < M (x passes)
};

__device__ __forceinline__ bool pred_ok(int pred, const ItemState& s, const ItemParams& p) {
  switch (pred) {
    case P_ACTIVE: return !s.done;
    case P_EXIT: return s.done && s.t >= 1;
    case P_PRECLIP: return __longlong_as_double((long long)s.emaxbits) > p.E;
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
template <typename T, int L>
struct Geo {
  static constexpr int W = 64 / (int)sizeof(v2<T>);   // pencils per tile
  static constexpr int NT = L / 8;                     // threads per pencil
  static constexpr int TPT = NT * W;                   // threads per tile
  static constexpr int G = TPT >= 256 ? 1 : 256 / TPT; // tiles per CTA
  static constexpr int NTHR = G * TPT;
  static constexpr int TILE_ELEMS = L * W;
  static constexpr int MINB = sizeof(T) == 4 ? (1024 / NTHR > 0 ? 1024 / NTHR : 1)
                                             : (512 / NTHR > 0 ? 512 / NTHR : 1);
};

// Block reduction of (max, count, sum, nan flag); thread 0 publishes.
struct Red {
  double vmax;
  double sum;
  unsigned long long cnt;
  int nan;
};
__device__ __forceinline__ void block_reduce(Red& r, double* sm_d, unsigned long long* sm_c,
                                             int* sm_n) {
  const unsigned full = 0xffffffffu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r.vmax = fmax(r.vmax, __shfl_xor_sync(full, r.vmax, o));
    r.sum += __shfl_xor_sync(full, r.sum, o);
    r.cnt += __shfl_xor_sync(full, r.cnt, o);
    r.nan |= __shfl_xor_sync(full, r.nan, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) { sm_d[wid] = r.vmax; sm_d[32 + wid] = r.sum; sm_c[wid] = r.cnt; sm_n[wid] = r.nan; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < nw; ++i) {
      r.vmax = fmax(r.vmax, sm_d[i]); r.sum += sm_d[32 + i]; r.cnt += sm_c[i]; r.nan |= sm_n[i];
    }
  }
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long* p, double v) {
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__device__ __forceinline__ T clampT(T x, T b) { return x > b ? b : (x < -b ? -b : x); }

// ---------------------------------------------------------------------------
// x passes: real rows <-> packed complex rows (R2C / C2R of length Nx = 2M
// through one length-M complex FFT of z[n] = r[2n] + i r[2n+1]).
// ---------------------------------------------------------------------------

// Post-processing of Z = FFT_M(z) into the packed half spectrum P (in place
// in registers).  Needs Z[M-k]; it is fetched from the tile in shared memory.
template <typename T, int M>
__device__ __forceinline__ void r2c_post(v2<T> (&v)[8], int j, const Slot<T>& sm,
                                         const v2<T>* __restrict__ twr) {
  constexpr int NT = M / 8;
#pragma unroll
  for (int u = 0; u < 8; ++u) sm.at(j + u * NT) = v[u];
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int k = j + u * NT;
    const v2<T> zk = v[u];
    const v2<T> zm = sm.at((M - k) & (M - 1));
    if (k == 0) {
      v[u] = mk<T>(zk.x + zk.y, zk.x - zk.y);
    } else {
      // Fe = (Zk + conj Zm)/2, Fo = (Zk - conj Zm)/(2i), X = Fe + W^k Fo
      const v2<T> fe = mk<T>(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
      const v2<T> fo = mk<T>(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x));
      v[u] = add<T>(fe, cmul<T>(twr[k], fo));
    }
  }
  __syncthreads();
}

// Pre-processing of packed P into Z' = 2 Z so that IFFT_M(Z') / Nx gives
// the real row (again one exchange for P[M-k]).
template <typename T, int M>
__device__ __forceinline__ void c2r_pre(v2<T> (&v)[8], int j, const Slot<T>& sm,
                                        const v2<T>* __restrict__ twr) {
  constexpr int NT = M / 8;
#pragma unroll
  for (int u = 0; u < 8; ++u) sm.at(j + u * NT) = v[u];
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int k = j + u * NT;
    const v2<T> xk = v[u];
    const v2<T> xm = sm.at((M - k) & (M - 1));
    if (k == 0) {
      v[u] = mk<T>(xk.x + xk.y, xk.x - xk.y);
    } else {
      // Z' = (Xk + conj Xm) + i (Xk - conj Xm) conj(W^k)
      const v2<T> s = mk<T>(xk.x + xm.x, xk.y - xm.y);
      const v2<T> d = cmulc<T>(mk<T>(xk.x - xm.x, xk.y + xm.y), twr[k]);
      v[u] = mk<T>(s.x - d.y, s.y + d.x);
    }
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ void load_tables(v2<T>* s_tw, const void* tw, int L, v2<T>* s_twr,
                                            const void* twr, int M) {
  const v2<T>* gtw = reinterpret_cast<const v2<T>*>(tw);
  for (int i = threadIdx.x; i < L; i += blockDim.x) s_tw[i] = gtw[i];
  if (s_twr) {
    const v2<T>* gtr = reinterpret_cast<const v2<T>*>(twr);
    for (int i = threadIdx.x; i < M; i += blockDim.x) s_twr[i] = gtr[i];
  }
}

// Shared-memory carve-up: [tiles][twiddles][R2C twiddles][reduction scratch].
template <typename T, int L>
struct Smem {
  static constexpr size_t tiles = (size_t)Geo<T, L>::G * Geo<T, L>::TILE_ELEMS * sizeof(v2<T>);
  static constexpr size_t tw = (size_t)L * sizeof(v2<T>);
  static constexpr size_t red = 32 * 8 * 2 + 32 * 8 + 32 * 4;
  static constexpr size_t bytes_axis = tiles + tw + red;
  static constexpr size_t bytes_x = tiles + 2 * tw + red;
};

// Entry / certification x pass: float32 real rows -> packed spectrum.
template <typename T, int M>
__global__ void __launch_bounds__(Geo<T, M>::NTHR, Geo<T, M>::MINB)
k_xfwd(Args a) {
  using G_ = Geo<T, M>;
  extern __shared__ __align__(16) unsigned char smraw[];
  v2<T>* s_tiles = reinterpret_cast<v2<T>*>(smraw);
  v2<T>* s_tw = s_tiles + G_::G * G_::TILE_ELEMS;
  v2<T>* s_twr = s_tw + M;
  double* s_red = reinterpret_cast<double*>(s_twr + M);

  const int gi = blockIdx.y;
  const int item = a.g.item[gi];
  const ItemParams& p = a.prm[item];
  ItemState& st = a.st[item];
  if (!pred_ok(a.pred, st, p)) return;
  load_tables<T>(s_tw, a.tw, M, s_twr, a.twr, M);

  const int g = threadIdx.x / G_::TPT, tid = threadIdx.x % G_::TPT;
  const int w = tid % G_::W, j = tid / G_::W;
  const int64_t tile = (int64_t)blockIdx.x * G_::G + g;
  const int64_t ntiles = a.g.rows / G_::W;
  const bool live = tile < ntiles;
  const int64_t row = live ? tile * G_::W + w : 0;
  Slot<T> sm{s_tiles + g * G_::TILE_ELEMS, w};

  const float* src = (a.mode & M_MASK) ? a.ein : a.e;
  const float2* erow = reinterpret_cast<const float2*>(src + a.g.eoff[gi]) + row * M;
  float2* erow_w = reinterpret_cast<float2*>(a.e + a.g.eoff[gi]) + row * M;
  Red r{0.0, 0.0, 0ull, 0};
  uint32_t bits = 0;
  if ((a.mode & M_MASK) && live) bits = a.mask[tile * G_::TPT + tid];
  v2<T> v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    float2 x = erow[j + u * G_::NT];
    if (a.mode & M_MEASURE) {
      const double ax = fabs((double)x.x), ay = fabs((double)x.y);
      r.vmax = fmax(r.vmax, fmax(ax, ay));
      r.sum += (double)x.x * x.x + (double)x.y * x.y;
      r.nan |= (x.x != x.x) | (x.y != x.y);
    }
    if (a.mode & M_PRECLIP) {
      const float cx = clampT<float>(x.x, p.Esf), cy = clampT<float>(x.y, p.Esf);
      r.cnt += (cx != x.x) + (cy != x.y);
      x.x = cx; x.y = cy;
      if (live) erow_w[j + u * G_::NT] = x;
    }
    if (a.mode & M_MASK) {
      if (!((bits >> (2 * u)) & 1u)) x.x = 0.f;
      if (!((bits >> (2 * u + 1)) & 1u)) x.y = 0.f;
    }
    v[u] = mk<T>((T)x.x, (T)x.y);
  }
  if (!live) r = Red{0.0, 0.0, 0ull, 0};
  __syncthreads();
  fft_pencil<T, M, -1>(v, j, s_tw, sm);
  r2c_post<T, M>(v, j, sm, s_twr);
  if (live) {
    v2<T>* out = pick<T>(a, a.sel_out, st.t) + a.g.soff[gi] + row * M;
#pragma unroll
    for (int u = 0; u < 8; ++u) out[j + u * G_::NT] = v[u];
  }
  if (a.mode & (M_MEASURE | M_PRECLIP)) {
    block_reduce(r, s_red, reinterpret_cast<unsigned long long*>(s_red + 64),
                 reinterpret_cast<int*>(s_red + 96));
    if (threadIdx.x == 0) {
      if (a.mode & M_MEASURE) {
        atomic_max_pos(&st.emaxbits, r.nan ? INFINITY : r.vmax);
        atomicAdd(&st.sumsq, r.sum);
      }
      if ((a.mode & M_PRECLIP) && r.cnt) atomicAdd(&st.act_s, r.cnt);
    }
  }
}

// Loop body x pass: C2R, scale 1/N, s-clip (or adjoint mask), R2C.
template <typename T, int M>
__global__ void __launch_bounds__(Geo<T, M>::NTHR, Geo<T, M>::MINB)
k_px(Args a) {
  using G_ = Geo<T, M>;
  extern __shared__ __align__(16) unsigned char smraw[];
  v2<T>* s_tiles = reinterpret_cast<v2<T>*>(smraw);
  v2<T>* s_tw = s_tiles + G_::G * G_::TILE_ELEMS;
  v2<T>* s_twr = s_tw + M;
  double* s_red = reinterpret_cast<double*>(s_twr + M);

  const int gi = blockIdx.y;
  const int item = a.g.item[gi];
  const ItemParams& p = a.prm[item];
  ItemState& st = a.st[item];
  if (!pred_ok(a.pred, st, p)) return;
  load_tables<T>(s_tw, a.tw, M, s_twr, a.twr, M);
  const int t = st.t;

  const int g = threadIdx.x / G_::TPT, tid = threadIdx.x % G_::TPT;
  const int w = tid % G_::W, j = tid / G_::W;
  const int64_t tile = (int64_t)blockIdx.x * G_::G + g;
  const int64_t ntiles = a.g.rows / G_::W;
  const bool live = tile < ntiles;
  const int64_t row = live ? tile * G_::W + w : 0;
  Slot<T> sm{s_tiles + g * G_::TILE_ELEMS, w};

  const v2<T>* in = pick<T>(a, a.sel_in, t) + a.g.soff[gi] + row * M;
  v2<T> v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) v[u] = in[j + u * G_::NT];
  __syncthreads();
  c2r_pre<T, M>(v, j, sm, s_twr);
  fft_pencil<T, M, +1>(v, j, s_tw, sm);

  Red r{0.0, 0.0, 0ull, 0};
  uint32_t bits = 0;
  const bool ck = (a.mode & M_CKPT) && a.ckpt_every > 0 && (t % a.ckpt_every) == 0;
  float2* ck_row = ck ? reinterpret_cast<float2*>(a.ckpt + (int64_t)(t / a.ckpt_every) * (2 * M * a.g.rows)) + row * M
                      : nullptr;
  if ((a.mode & M_MASK) && live) bits = a.mask[tile * G_::TPT + tid];
  const T inv_n = sizeof(T) == 4 ? (T)p.inv_nf : (T)p.inv_n;
  const T Es = sizeof(T) == 4 ? (T)p.Esf : (T)p.Es;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    T x = v[u].x * inv_n, y = v[u].y * inv_n;
    if (a.mode & M_CLIP) {
      const T cx = clampT<T>(x, Es), cy = clampT<T>(y, Es);
      const bool ix = (cx == x), iy = (cy == y);   // inside the s-cube
      r.cnt += (!ix) + (!iy);
      bits |= ((uint32_t)ix << (2 * u)) | ((uint32_t)iy << (2 * u + 1));
      x = cx; y = cy;
      if (ck && live) ck_row[j + u * G_::NT] = make_float2((float)x, (float)y);
    } else if (a.mode & M_MASK) {
      if (!((bits >> (2 * u)) & 1u)) x = T(0);
      if (!((bits >> (2 * u + 1)) & 1u)) y = T(0);
    }
    v[u] = mk<T>(x, y);
  }
  if ((a.mode & M_RECORD) && live) a.mask[tile * G_::TPT + tid] = bits;
  fft_pencil<T, M, -1>(v, j, s_tw, sm);
  r2c_post<T, M>(v, j, sm, s_twr);
  if (live) {
    v2<T>* out = pick<T>(a, a.sel_out, t) + a.g.soff[gi] + row * M;
#pragma unroll
    for (int u = 0; u < 8; ++u) out[j + u * G_::NT] = v[u];
  }
  if (a.mode & M_CLIP) {
    if (!live) r.cnt = 0;
    block_reduce(r, s_red, reinterpret_cast<unsigned long long*>(s_red + 64),
                 reinterpret_cast<int*>(s_red + 96));
    if (threadIdx.x == 0 && r.cnt) atomicAdd(&st.act_s, r.cnt);
  }
}

// Exit x pass: C2R, scale 1/N, s-clip, store float32 e (rebuilds the iterate
// e_t from the input of the last loop body).  In mask mode (adjoint exit)
// no clip is applied.
template <typename T, int M>
__global__ void __launch_bounds__(Geo<T, M>::NTHR, Geo<T, M>::MINB)
k_xexit(Args a) {
  using G_ = Geo<T, M>;
  extern __shared__ __align__(16) unsigned char smraw[];
  v2<T>* s_tiles = reinterpret_cast<v2<T>*>(smraw);
  v2<T>* s_tw = s_tiles + G_::G * G_::TILE_ELEMS;
  v2<T>* s_twr = s_tw + M;

  const int gi = blockIdx.y;
  const int item = a.g.item[gi];
  const ItemParams& p = a.prm[item];
  ItemState& st = a.st[item];
  if (!pred_ok(a.pred, st, p)) return;
  load_tables<T>(s_tw, a.tw, M, s_twr, a.twr, M);
  const int t = st.t;

  const int g = threadIdx.x / G_::TPT, tid = threadIdx.x % G_::TPT;
  const int w = tid % G_::W, j = tid / G_::W;
  const int64_t tile = (int64_t)blockIdx.x * G_::G + g;
  const int64_t ntiles = a.g.rows / G_::W;
  const bool live = tile < ntiles;
  const int64_t row = live ? tile * G_::W + w : 0;
  Slot<T> sm{s_tiles + g * G_::TILE_ELEMS, w};

  const v2<T>* in = pick<T>(a, a.sel_in, t) + a.g.soff[gi] + row * M;
  v2<T> v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) v[u] = in[j + u * G_::NT];
  __syncthreads();
  c2r_pre<T, M>(v, j, sm, s_twr);
  fft_pencil<T, M, +1>(v, j, s_tw, sm);
  const T inv_n = sizeof(T) == 4 ? (T)p.inv_nf : (T)p.inv_n;
  const T Es = sizeof(T) == 4 ? (T)p.Esf : (T)p.Es;
  float2* erow = reinterpret_cast<float2*>(a.e + a.g.eoff[gi]) + row * M;
  if (live) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      T x = v[u].x * inv_n, y = v[u].y * inv_n;
      if (a.mode & M_CLIP) { x = clampT<T>(x, Es); y = clampT<T>(y, Es); }
      float fx = (float)x, fy = (float)y;
      if (a.mode & M_CLIP) {
        // keep the float32 result inside the shrunk cube after rounding
        fx = clampT<float>(fx, p.Esf); fy = clampT<float>(fy, p.Esf);
      }
      erow[j + u * G_::NT] = make_float2(fx, fy);
    }
  }
}

// ---------------------------------------------------------------------------
// Strided axis passes
// ---------------------------------------------------------------------------

// Plain C2C along the middle axis of a 3D item (y): pencils at fixed (z, kx).
template <typename T, int L, int DIR>
__global__ void __launch_bounds__(Geo<T, L>::NTHR, Geo<T, L>::MINB)
k_axis(Args a) {
  using G_ = Geo<T, L>;
  extern __shared__ __align__(16) unsigned char smraw[];
  v2<T>* s_tiles = reinterpret_cast<v2<T>*>(smraw);
  v2<T>* s_tw = s_tiles + G_::G * G_::TILE_ELEMS;

  const int gi = blockIdx.y;
  const int item = a.g.item[gi];
  const ItemParams& p = a.prm[item];
  ItemState& st = a.st[item];
  if (!pred_ok(a.pred, st, p)) return;
  load_tables<T>(s_tw, a.tw, L, nullptr, nullptr, 0);
  const int t = st.t;

  const int g = threadIdx.x / G_::TPT, tid = threadIdx.x % G_::TPT;
  const int w = tid % G_::W, j = tid / G_::W;
  const int M = a.g.M;
  const int tpr = M / G_::W;                      // tiles per z-plane
  const int64_t tile = (int64_t)blockIdx.x * G_::G + g;
  const int64_t ntiles = (int64_t)a.g.Nz * tpr;
  const bool live = tile < ntiles;
  const int64_t z = live ? tile / tpr : 0;
  const int kx = live ? (int)(tile % tpr) * G_::W + w : 0;
  const int64_t base = a.g.soff[gi] + z * (int64_t)L * M + kx;
  Slot<T> sm{s_tiles + g * G_::TILE_ELEMS, w};

  const v2<T>* in = pick<T>(a, a.sel_in, t) + base;
  v2<T> v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) v[u] = in[(int64_t)(j + u * G_::NT) * M];
  __syncthreads();
  fft_pencil<T, L, DIR>(v, j, s_tw, sm);
  if (live) {
    v2<T>* out = pick<T>(a, a.sel_out, t) + base;
#pragma unroll
    for (int u = 0; u < 8; ++u) out[(int64_t)(j + u * G_::NT) * M] = v[u];
  }
}

// Check / f-clip pass along the outermost axis (z in 3D, y in 2D): forward
// FFT completes the spectrum; the violation max over all bins is reduced
// (CheckConvergence), Re and Im are clipped to +-D' (ProjectOntoFCube), and
// the inverse FFT of this axis is applied before the store.
//
// Tiles are of two kinds.  Main tiles: W consecutive kx >= 1 at one middle
// index (slot kx = 0 skipped).  Mirror tiles: the kx = 0 pencils, in pairs
// (m, -m) of middle indices so that A and B can be separated; a pencil that
// is its own mirror (m = 0 or Nmid/2) fills both slots of its pair and only
// the first slot stores.
template <typename T, int L>
__global__ void __launch_bounds__(Geo<T, L>::NTHR, Geo<T, L>::MINB)
k_chk(Args a) {
  using G_ = Geo<T, L>;
  constexpr int W = G_::W, NT = G_::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  v2<T>* s_tiles = reinterpret_cast<v2<T>*>(smraw);
  v2<T>* s_tw = s_tiles + G_::G * G_::TILE_ELEMS;
  double* s_red = reinterpret_cast<double*>(s_tw + L);

  const int gi = blockIdx.y;
  const int item = a.g.item[gi];
  const ItemParams& p = a.prm[item];
  ItemState& st = a.st[item];
  if (!pred_ok(a.pred, st, p)) return;
  load_tables<T>(s_tw, a.tw, L, nullptr, nullptr, 0);
  const int t = st.t;

  const int g = threadIdx.x / G_::TPT, tid = threadIdx.x % G_::TPT;
  const int w = tid % W, j = tid / W;
  const int M = a.g.M, Nmid = a.g.Nmid;
  const int tpr = M / W;
  const int64_t nmain = (int64_t)Nmid * tpr;
  const int npairs = Nmid / 2 + 1;   // pairs (m, -m), m = 0..Nmid/2
  const int64_t nmirror = (npairs + W / 2 - 1) / (W / 2);
  const int64_t tile = (int64_t)blockIdx.x * G_::G + g;
  const bool live = tile < nmain + nmirror;
  const bool mirror = live && tile >= nmain;
  const int64_t estride = (int64_t)Nmid * M;

  int64_t base = 0;
  bool owner = false, valid = false;
  if (live && !mirror) {
    const int mid = (int)(tile / tpr);
    const int kx = (int)(tile % tpr) * W + w;
    base = (int64_t)mid * M + kx;
    valid = kx != 0;
    owner = valid;
  } else if (mirror) {
    const int q = (int)(tile - nmain) * (W / 2) + (w >> 1);
    const int m = w & 1;
    const int nh = Nmid / 2;
    valid = q < npairs;
    const bool selfm = (q == 0) || (q == nh);
    const int mid = !valid ? 0 : (selfm ? q : (m ? Nmid - q : q));
    base = (int64_t)mid * M;
    owner = valid && (m == 0 || !selfm);
  }
  Slot<T> sm{s_tiles + g * G_::TILE_ELEMS, w};

  v2<T>* buf = pick<T>(a, a.sel_in, t) + a.g.soff[gi] + base;
  v2<T> v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) v[u] = buf[(int64_t)(j + u * NT) * estride];
  __syncthreads();
  fft_pencil<T, L, -1>(v, j, s_tw, sm);

  // Any tile of this CTA may be a mirror tile; the exchange below needs the
  // whole CTA, so it runs whenever one of the CTA's tiles is.
  const int64_t first_tile = (int64_t)blockIdx.x * G_::G;
  const int64_t last_tile = first_tile + G_::G - 1;
  const bool cta_has_mirror = last_tile >= nmain && first_tile < nmain + nmirror;

  const T Ds = sizeof(T) == 4 ? (T)p.Dsf : (T)p.Ds;
  Red r{0.0, 0.0, 0ull, 0};
  uint32_t bits = 0;
  const bool rec = (a.mode & M_RECORD) != 0, use_mask = (a.mode & M_MASK) != 0;
  if (use_mask && live) bits = a.mask[tile * G_::TPT + tid];
  T vloc = T(0);
  if (cta_has_mirror) {
#pragma unroll
    for (int u = 0; u < 8; ++u) sm.at(j + u * NT) = v[u];
    __syncthreads();
    const Slot<T> smm{sm.base, w ^ 1};
    if (mirror) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const v2<T> c = v[u], m = smm.at((L - (j + u * NT)) & (L - 1));
        // A = (C + conj Cm)/2, B = (C - conj Cm)/(2i)
        T ar = T(0.5) * (c.x + m.x), ai = T(0.5) * (c.y - m.y);
        T br = T(0.5) * (c.y + m.y), bi = T(0.5) * (m.x - c.x);
        if (valid) {
          vloc = fmax(vloc, fmax(fmax(fabs(ar), fabs(ai)), fmax(fabs(br), fabs(bi))));
          r.nan |= (ar != ar) | (ai != ai) | (br != br) | (bi != bi);
        }
        if (a.mode & M_CLIP) {
          const T car = clampT<T>(ar, Ds), cai = clampT<T>(ai, Ds);
          const T cbr = clampT<T>(br, Ds), cbi = clampT<T>(bi, Ds);
          const bool iar = car == ar, iai = cai == ai, ibr = cbr == br, ibi = cbi == bi;
          if (owner) r.cnt += (!(iar && iai)) + (!(ibr && ibi));
          bits |= ((uint32_t)iar | ((uint32_t)iai << 1) | ((uint32_t)ibr << 2) | ((uint32_t)ibi << 3))
                  << (4 * u);
          ar = car; ai = cai; br = cbr; bi = cbi;
        } else if (use_mask) {
          const uint32_t b4 = bits >> (4 * u);
          if (!(b4 & 1u)) ar = T(0);
          if (!(b4 & 2u)) ai = T(0);
          if (!(b4 & 4u)) br = T(0);
          if (!(b4 & 8u)) bi = T(0);
        }
        v[u] = mk<T>(ar - bi, ai + br);   // C' = A' + i B'
      }
    }
    __syncthreads();
  }
  if (!mirror) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      T x = v[u].x, y = v[u].y;
      if (valid) {
        vloc = fmax(vloc, fmax(fabs(x), fabs(y)));
        r.nan |= (x != x) | (y != y);
      }
      if (a.mode & M_CLIP) {
        const T cx = clampT<T>(x, Ds), cy = clampT<T>(y, Ds);
        const bool ix = cx == x, iy = cy == y;
        if (owner) r.cnt += 2 * (!(ix && iy));   // a stored bin stands for k and -k
        bits |= ((uint32_t)ix << (2 * u)) | ((uint32_t)iy << (2 * u + 1));
        x = cx; y = cy;
      } else if (use_mask) {
        if (!((bits >> (2 * u)) & 1u)) x = T(0);
        if (!((bits >> (2 * u + 1)) & 1u)) y = T(0);
      }
      v[u] = mk<T>(x, y);
    }
  }
  if (rec && live) a.mask[tile * G_::TPT + tid] = bits;
  r.vmax = (double)vloc;
  if (!(a.mode & M_MASK)) {
    block_reduce(r, s_red, reinterpret_cast<unsigned long long*>(s_red + 64),
                 reinterpret_cast<int*>(s_red + 96));
    if (threadIdx.x == 0) {
      atomic_max_pos(&st.vbits, r.nan ? INFINITY : r.vmax);
      if (r.cnt) atomicAdd(&st.act_f, r.cnt);
    }
  }
  if (a.mode & M_NOWRITE) return;
  __syncthreads();
  fft_pencil<T, L, +1>(v, j, s_tw, sm);
  if (owner) {
    v2<T>* out = pick<T>(a, a.sel_out, t) + a.g.soff[gi] + base;
#pragma unroll
    for (int u = 0; u < 8; ++u) out[(int64_t)(j + u * NT) * estride] = v[u];
  }
}

// ---------------------------------------------------------------------------
// Per-item control kernels
// ---------------------------------------------------------------------------

// Loop decision after a check (Alg. 1: break when CheckConvergence passes;
// readings: stop at v <= D(1 - eta/2) once t >= min_iters, cap at max_iters).
__global__ void k_decide(const ItemParams* prm, ItemState* st, int n, int* n_active) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ItemState& s = st[i];
  if (s.done) return;
  const ItemParams& p = prm[i];
  const double v = __longlong_as_double((long long)s.vbits);
  s.vbits = 0ull;
  s.f_ratio = v / p.D;
  s.last_act_s = s.act_s;
  s.last_act_f = s.prev_act_f;
  s.prev_act_f = s.act_f;
  s.act_s = 0ull;
  s.act_f = 0ull;
  int done = 0;
  if (!(v <= DBL_MAX)) { done = 1; s.status = 6; }
  else if (v <= p.thr && s.t >= p.min_iters) { done = 1; s.status = 0; }
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
__global__ void k_init(ItemState* st, int n, int only_uncertified, int* n_active) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ItemState& s = st[i];
  const bool run = !only_uncertified || !s.certified;
  s.vbits = 0ull; s.emaxbits = 0ull; s.sumsq = 0.0;
  s.act_s = s.act_f = 0ull; s.last_act_s = s.last_act_f = s.prev_act_f = 0ull;
  s.t = 0;
  s.done = run ? 0 : 1;
  if (!only_uncertified) { s.status = 0; s.preclip = 0; s.certified = 0; s.repairs = 0; s.f_ratio = 0.0; }
  if (run) atomicAdd(n_active, 1);
}

__global__ void k_mark_preclip(const ItemParams* prm, ItemState* st, int n) {
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
__global__ void k_certify(const ItemParams* prm, ItemState* st, int n, int repair_round) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ItemState& s = st[i];
  const ItemParams& p = prm[i];
  if (repair_round && s.certified) return;
  const double emax = __longlong_as_double((long long)s.emaxbits);
  const double v = __longlong_as_double((long long)s.vbits);
  const double ln = log2((double)p.n);
  const double b = 10.0 * (ln + 2.0) * 1.1102230246251565e-16 * sqrt((double)p.n * s.sumsq);
  s.v64 = v;
  s.emax64 = emax;
  s.bound64 = b;
  s.certified = (emax <= p.E) && (v + b <= p.D);
  s.vbits = 0ull;
  s.emaxbits = 0ull;
  s.sumsq = 0.0;
}

// g <- g * [|e0| <= E'] for items whose input was pre-clipped (adjoint of
// the pre-loop s-projection).
__global__ void k_premask(float* g, const float* e0, const ItemParams* prm, const ItemState* st,
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
