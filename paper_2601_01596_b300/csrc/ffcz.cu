// ffcz.cu -- plan, executor and C ABI of the FFCz correction library.
//
// Host side of the hot path of Alg. 1 (Sec. IV-B) and its GPU mapping
// (Sec. IV-D): every step runs in the kernels of passes.cuh; the host only
// sequences launches, replays loop chunks as CUDA graphs and reads one
// 4-byte "items still running" counter between chunks.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/ffcz.h"
#include "bluestein.cuh"
#include "passes.cuh"
#include "edits.cuh"
#include "multi.cuh"

using namespace ffcz;

namespace {

thread_local std::string g_err;
std::atomic<int64_t> g_launches{0};

struct Fail {
  ffcz_status s;
};

void fail(ffcz_status s, const std::string& msg) {
  g_err = msg;
  throw Fail{s};
}

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      fail(e_ == cudaErrorMemoryAllocation ? FFCZ_ERR_OOM : FFCZ_ERR_CUDA,        \
           std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    }                                                                             \
  } while (0)

bool is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

// exp(-2 pi i m / L) in long double (exact zeros kept exact).
void root_ld(long double m, long double L, long double& c, long double& s) {
  static const long double pi = acosl(-1.0L);
  const long double a = 2.0L * pi * m / L;
  c = cosl(a);
  s = -sinl(a);
  if (fabsl(c) < 1e-18L) c = 0.0L;
  if (fabsl(s) < 1e-18L) s = 0.0L;
}

// exp(-2 pi i m / L) rounded once to T.
template <typename T>
v2<T> root(long double m, long double L) {
  long double c, s;
  root_ld(m, L, c, s);
  v2<T> r;
  r.x = (T)c;
  r.y = (T)s;
  return r;
}

// exp(-2 pi i k / Nx) for k < Nx/2 (R2C / C2R post- and pre-processing).
template <typename T>
std::vector<v2<T>> r2c_table(int Nx) {
  std::vector<v2<T>> t(Nx / 2);
  for (int k = 0; k < Nx / 2; ++k) t[k] = root<T>(k, Nx);
  return t;
}

// Stage-2 twiddles of the two-stage split of L (layout in fft_core.cuh):
// exp(-2 pi i k1 t / L), k1 < R1, t = 1..R2-1, at tw_index(R1, k1, t).
template <typename T>
std::vector<v2<T>> stage_table_rt(int L, int S = 0) {
  const int R1 = split_r1(L, S), R2 = L / R1;
  std::vector<v2<T>> t(L);
  for (auto& x : t) { x.x = 0; x.y = 0; }
  for (int k1 = 0; k1 < R1; ++k1)
    for (int tt = 1; tt < R2; ++tt) {
      if constexpr (sizeof(T) == 8) {
        // FP64: factors tt >= R2/2 in the tangent form of the fused layer
        long double c, sn;
        root_ld((long double)k1 * tt, (long double)L, c, sn);
        t[tw_index(R1, k1, tt)] = f64_stage_entry(c, sn, tt >= R2 / 2);
      } else {
        t[tw_index(R1, k1, tt)] = root<T>((long double)k1 * tt, (long double)L);
      }
    }
  return t;
}

struct DevGroup {
  Group g;            // device pointers inside
  int count;
  int ndim, Nz, Ny, Nx, M;
  int64_t rows, n;
  // float32 tile widths (pencils per tile) picked by the tuner per pass kind:
  // strided passes (y, chk, 1D column) 4 or 8; contiguous passes (x, 1D
  // row) 32/NT or 64/NT (a tile of one or two warps); set at plan creation
  int wx = 0, wa = 8, wc = 8, w1c = 8, w1r = 0;
  // TMA tensor maps of the float32 spectrum buffers (device arrays of
  // 2 x count maps, [2 gi + buffer]) for the y pass and the check pass;
  // null where the TMA-fed kernels do not apply
  const CUtensorMap* tm_axis = nullptr;
  const CUtensorMap* tm_chk = nullptr;
  // the check pass's view of its auxiliary packed field, the pointwise
  // f-bounds or the variants' residual (count maps)
  const CUtensorMap* tm_aux = nullptr;
  std::vector<int64_t> h_soff;   // host copy of the members' spectrum offsets
  const int64_t* d_canon = nullptr;   // members' offsets in the canonical edit spectra
  // 1D items (Bluestein): P = P1 P2 >= 2N - 1; exp(-2 pi i m / P) tables
  int P1 = 0, P2 = 0;
  const void* twp32 = nullptr;
  const void* twp64 = nullptr;
};

struct Tables {
  // per power of two 2^p: stage-2 twiddles (p = 3..10) and R2C
  // factors for Nx = 2^p (p = 4..11)
  void* f32[12] = {};
  void* f64[12] = {};
  void* r32[12] = {};
  void* r64[12] = {};
  // stage factors of the swapped radix split (odd p; fft_core.cuh Split)
  void* f32s[12] = {};
  void* f64s[12] = {};
};

template <typename T>
const void* tw_of(const Tables& tb, int L) {
  const int p = ilog2(L);
  return sizeof(T) == 4 ? tb.f32[p] : tb.f64[p];
}
template <typename T>
const void* tw1_of(const Tables& tb, int L) {
  const int p = ilog2(L);
  return sizeof(T) == 4 ? tb.f32s[p] : tb.f64s[p];
}
// The stage tables of a pass of length L in both radix splits.
template <typename T>
void set_tw(Args& a, const Tables& tb, int L) {
  a.tw = tw_of<T>(tb, L);
  a.tw1 = tw1_of<T>(tb, L);
}
template <typename T>
const void* twr_of(const Tables& tb, int Nx) {
  const int p = ilog2(Nx);
  return sizeof(T) == 4 ? tb.r32[p] : tb.r64[p];
}

}  // namespace

struct ffcz_plan_s {
  int ndim = 0;
  int64_t batch = 0;
  std::vector<int64_t> shapes;
  std::vector<int64_t> eoff;   // float offset per item
  int64_t total = 0;           // floats
  int64_t total_c = 0;         // complex values per spectrum buffer
  ffcz_opts opts{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;   // private stream used only to capture graphs
  cudaStream_t copy_stream = nullptr;  // host-buffer entry point: copy-back stream
  cudaEvent_t ev_copy = nullptr;
  // host-buffer entry point: the upload in row chunks and the FP64 x pass
  // (3D: and y pass) on each chunk as it lands (spec_stream), into a side
  // state d_stc; spec_y: the y pass ran too
  cudaStream_t spec_stream = nullptr;
  std::vector<cudaEvent_t> ev_chunks;
  cudaEvent_t ev_spec = nullptr;
  ItemState* d_stc = nullptr;
  bool spec_y = false;
  int device = 0;

  std::vector<DevGroup> groups;
  std::vector<void*> allocs;
  Tables tb;

  void* B32[2] = {nullptr, nullptr};
  void* Bt32 = nullptr;        // 1D: FFT_P of the wrapped chirps (float32 / float64)
  void* Bt64 = nullptr;
  void* ch32 = nullptr;        // 1D: chirp tables b_n (float32 / float64)
  void* ch64 = nullptr;
  // 1D certification of even lengths through the N/2-point transform of
  // x_2n + i x_2n+1: groups of the P/2-point passes, the N/2-point chirps and
  // their Bt, the spectrum Z and the twiddles W_N^k (built at the first
  // certification)
  std::vector<DevGroup> hgroups;
  void* ch64h = nullptr;
  void* Bt64h = nullptr;
  void* Bz = nullptr;
  double2* rtw = nullptr;
  void* B64[2] = {nullptr, nullptr};
  void* Bc = nullptr;
  float* staging = nullptr;
  ItemParams* d_prm = nullptr;
  ItemState* d_st = nullptr;
  ItemState* d_st2 = nullptr;   // adjoint state
  int* d_nactive = nullptr;
  int* h_nactive = nullptr;     // pinned
  int* d_err = nullptr;         // device error word (DevErr), cleared per call
  // Alg. 1 edits (opts.edits): spatial edits (float32, like e), frequency
  // edits in the packed spectrum layout (committed, pending, pending tag),
  // recorded only by the correction loops (ed_on), plus the canonical
  // half-spectrum form and compaction scratch built on request
  float* ed_s = nullptr;
  float2* ed_f = nullptr;
  float2* ed_p = nullptr;
  int* ed_t = nullptr;
  bool ed_on = false;
  float2* ed_canon = nullptr;
  int* ed_chunks = nullptr;
  // pointwise bounds (opts.pointwise): copies of the caller's E_n and Delta_k
  float* pw_e = nullptr;
  float2* pw_f = nullptr;
  float2* pw_fp = nullptr;          // the same in the packed spectrum layout
  float4* pw_f0 = nullptr;          // per x-row: bounds of the kx = 0 and Nx/2 planes
  int64_t total_rows = 0;
  unsigned int* pw_min = nullptr;   // per item min Delta (float bits)
  int* pw_bad = nullptr;
  // projection variant (opts.method): residual spectrum and the two
  // parity buffers of q / u, used by the float32 loop only (pv_on)
  float2* pv_r = nullptr;
  float* pv_q[2] = {nullptr, nullptr};
  bool pv_on = false;
  double* ps_acc = nullptr;         // power-spectrum shell sums (3 S per item)
  double* ps_rho = nullptr;
  int ps_S = 0;
  // per item: points, half-spectrum bins, and the offsets of its regions in
  // the caller's edit arrays (spatial flags/codes, frequency flags/codes)
  std::vector<std::array<int64_t, 6>> ed_layout;
  std::array<int64_t, 6> ed_total{};
  void* ed_reg_s = nullptr;      // device EdRegion<float>[batch]
  void* ed_reg_f = nullptr;      // device EdRegion<float2>[batch]
  int64_t* ed_tot = nullptr;     // device per-region counts [2 batch]
  void* ap_reg = nullptr;        // device ApRegion[2 batch] (edit application)
  int64_t ed_chunk_cap = 0;
  // 16-bit code storage: int32 codes of every region, code regions, escape
  // counts, chunk offsets
  int32_t* cd_c32 = nullptr;
  void* cd_reg = nullptr;        // device CodeRegion[2 batch]
  int64_t* cd_tot = nullptr;     // device [2 batch]
  int* cd_chunks = nullptr;
  int64_t cd_chunk_cap = 0;
  int* h_err = nullptr;         // pinned copy
  int num_sms = 148;
  ItemState* h_st = nullptr;    // pinned
  ItemParams* h_prm = nullptr;  // pinned
  size_t ws_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;

  // graphs of loop chunks: key = (precision, chunk); the device-side WHILE
  // loop graph: key = (-precision, 0)
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
  std::map<std::pair<int, int>, int> graph_nodes;
  int* d_loopcount = nullptr;   // bodies executed by the WHILE graph
  int* h_loopcount = nullptr;   // pinned copy
  bool count_pending = false;
  // [precision][checkpoint recording + 2 x mask keeping]
  int while_cap[2][4] = {{-1, -1, -1, -1}, {-1, -1, -1, -1}};
  int pending_bodies_per = 0;

  // per-kernel profile (events around every launch; graphs off while on)
  bool prof = false;
  struct Pending { std::string key; cudaEvent_t a, b; };
  std::vector<Pending> pend;
  std::vector<cudaEvent_t> evpool;
  std::map<std::string, std::pair<double, int64_t>> prof_tab;
  std::vector<std::string> prof_keys;

  // multi-group form of the loop passes (one launch per pass kind over the
  // members of every shape group, multi.cuh): the work list of each kind,
  // the grid and shared memory of its launch, and whether the tuner took it
  struct MultiPlan { int2* units = nullptr; int64_t n = 0; int grid = 0; size_t smem = 0; };
  MultiPlan mp[MK_N];
  bool multi_use[MK_N] = {};

  // backward workspace
  float* bw_e = nullptr;
  float* bw_ck = nullptr;
  uint32_t* bw_smask = nullptr;
  uint32_t* bw_fmask = nullptr;
  void* bw_G[2] = {nullptr, nullptr};
  int bw_K = -1, bw_m = -1;
  // forward of the differentiable form: the loop's x pass writes the
  // backward's checkpoints into bw_ck (ffcz_correct_ckpt)
  bool ck_rec = false;
  // ffcz_correct_ckpt with opts.keep_masks: the masks of every step (x-pass
  // masks of step t at t px_words, check-pass masks of check t at t chk_words)
  uint32_t* km_s = nullptr;
  uint32_t* km_f = nullptr;
  int km_K = 0;
  bool km_valid = false;   // they describe the last ffcz_correct_ckpt call
  int64_t px_words = 0, chk_words = 0;       // mask words of one step (all groups)
  std::vector<int64_t> bw_pxoff, bw_chkoff;  // each group's offset in a step's block
};

namespace {

void* dalloc(ffcz_plan_s* p, size_t bytes) {
  void* ptr = nullptr;
  CK(cudaMalloc(&ptr, bytes));
  p->allocs.push_back(ptr);
  p->ws_bytes += bytes;
  return ptr;
}

template <typename Kern>
void set_smem(Kern k, size_t bytes) {
  if (bytes > 48 * 1024) CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

// When true, launch helpers only set kernel attributes (done once per plan,
// before any graph capture).
thread_local bool g_dry = false;

// Plan whose launches are being profiled on this thread (nullptr: none).
thread_local ffcz_plan_s* g_prof = nullptr;


cudaEvent_t prof_event(ffcz_plan_s* p) {
  if (!p->evpool.empty()) { cudaEvent_t e = p->evpool.back(); p->evpool.pop_back(); return e; }
  cudaEvent_t e;
  CK(cudaEventCreate(&e));
  return e;
}

struct ProfScope {
  ffcz_plan_s* p;
  cudaEvent_t a = nullptr;
  const char* kind;
  int prec, len;
  cudaStream_t s;
  ProfScope(const char* kind_, int prec_, int len_, cudaStream_t s_)
      : p(g_prof), kind(kind_), prec(prec_), len(len_), s(s_) {
    if (p) { a = prof_event(p); CK(cudaEventRecord(a, s)); }
  }
  ~ProfScope() noexcept(false) {
    if (!p) return;
    cudaEvent_t b = prof_event(p);
    CK(cudaEventRecord(b, s));
    char key[64];
    snprintf(key, sizeof key, "%s<f%d,%d>", kind, prec, len);
    p->pend.push_back({key, a, b});
  }
};

// Accumulate the elapsed times of all pending event pairs (stream is synced).
void prof_collect(ffcz_plan_s* p) {
  for (auto& x : p->pend) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, x.a, x.b));
    auto it = p->prof_tab.find(x.key);
    if (it == p->prof_tab.end()) {
      p->prof_keys.push_back(x.key);
      it = p->prof_tab.emplace(x.key, std::make_pair(0.0, (int64_t)0)).first;
    }
    it->second.first += ms;
    it->second.second += 1;
    p->evpool.push_back(x.a);
    p->evpool.push_back(x.b);
  }
  p->pend.clear();
}

// ----- kernel dispatch over the pencil length and the tile width -------------
// Strided float32 kernels exist with 4- and 8-pencil tiles, contiguous ones
// (rows along x, 1D rows) with tiles of one or two warps; the tuner picks per
// plan.  float64 kernels use 4-pencil strided tiles and one-warp rows.
// XCERT: the FP64 certification's x pass, which returns 2 X (exact; the
// certification halves its maximum) to save the multiplications by 1/2.
enum XKind { XFWD = 0, XPX = 1, XEXIT = 2, XCERT = 3 };

#define FFCZ_DISPATCH_L(Lv, FN, ...)                                     \
  switch (Lv) {                                                           \
    case 8: FN<8>(__VA_ARGS__); break;                                    \
    case 16: FN<16>(__VA_ARGS__); break;                                  \
    case 32: FN<32>(__VA_ARGS__); break;                                  \
    case 64: FN<64>(__VA_ARGS__); break;                                  \
    case 128: FN<128>(__VA_ARGS__); break;                                \
    case 256: FN<256>(__VA_ARGS__); break;                                \
    case 512: FN<512>(__VA_ARGS__); break;                                \
    case 1024: FN<1024>(__VA_ARGS__); break;                              \
    default: fail(FFCZ_ERR_UNSUPPORTED, "transform length");              \
  }

// Row-tile widths of a contiguous pass of length L: one warp, two warps.
constexpr int row_w1(int L) { return 32 / (1 << (ilog2(L) / 2)) > 0 ? 32 / (1 << (ilog2(L) / 2)) : 1; }
constexpr int row_w2(int L) { return 2 * row_w1(L); }

// Pointwise-bound plans select the PW kernel variants (the dry run sets
// g_pw_sel to reach them without bound pointers).
thread_local bool g_pw_sel = false;

// Width codes of the tuner: a plain kernel's tile width W, -W for the
// persistent copy-engine-fed kernel, and W | kSplit for the plain kernel in
// the swapped radix split (fft_core.cuh Split<L, 1>; odd log2 L only).
constexpr int kSplit = 256;
template <int L> constexpr bool split1_ok() { return ilog2(L) % 2 == 1; }

// The x pass needs its full form for edit recording and the adjoint's mask,
// record and checkpoint modes; every other launch takes the lean one.
inline bool px_full(const Args& a) { return (a.mode & (M_RECORD | M_MASK | M_CKPT)) != 0 || a.ed_s != nullptr; }

template <typename T, int M, int W, bool PW = false, int PV = PV_POCS, int S = 0>
void launch_x_tw(XKind kind, const Args& a, int64_t rows, int count, cudaStream_t s) {
  using G_ = Geo<T, M, W>;
  const int64_t tiles = (rows + G_::W - 1) / G_::W;
  dim3 grid((unsigned)((tiles + G_::G - 1) / G_::G), (unsigned)count);
  const size_t sm = Smem<T, M, W>::bytes_x;
  if (g_dry) {
    set_smem(k_xfwd<T, M, W, PW>, sm);
    if constexpr (sizeof(T) == 8) set_smem(k_xfwd<T, M, W, PW, true>, sm);
    if constexpr (PV == PV_POCS) set_smem(k_px<T, M, W, PW, PV, true>, sm);
    set_smem(k_px<T, M, W, PW, PV, false>, sm);
    if constexpr (S == 1) { set_smem(k_px<T, M, W, PW, PV, true, 1>, sm); set_smem(k_px<T, M, W, PW, PV, false, 1>, sm); }
    set_smem(k_xexit<T, M, W, PW, PV>, sm);
    return;
  }
  ProfScope ps(kind == XFWD || kind == XCERT ? "xfwd" : kind == XPX ? "px" : "xexit", 8 * (int)sizeof(T), M, s);
  switch (kind) {
    case XCERT:
      if constexpr (sizeof(T) == 8) { k_xfwd<T, M, W, PW, true><<<grid, G_::NTHR, sm, s>>>(a); break; }
      [[fallthrough]];
    case XFWD: k_xfwd<T, M, W, PW><<<grid, G_::NTHR, sm, s>>>(a); break;
    case XPX:
      // projection variants run lean only (no edits, no adjoint)
      if constexpr (PV == PV_POCS) {
        if (px_full(a)) { k_px<T, M, W, PW, PV, true, S><<<grid, G_::NTHR, sm, s>>>(a); break; }
      }
      k_px<T, M, W, PW, PV, false, S><<<grid, G_::NTHR, sm, s>>>(a);
      break;
    case XEXIT: k_xexit<T, M, W, PW, PV><<<grid, G_::NTHR, sm, s>>>(a); break;
  }
  g_launches++;
}
int g_num_sms_x = 148;   // set from the device at plan creation

// Persistent bulk-copy-fed loop x pass (float32, one-warp tiles): as many
// CTAs as fit on the device, spread over the group's items.
template <int M, bool ED, bool PW = false, int PV = PV_POCS>
void launch_px_tma_ed(const Args& a, int64_t rows, int count, cudaStream_t s) {
  constexpr int W = row_w1(M);
  using PG = PxTmaGeo<M, W>;
  const size_t sm = PG::bytes;
  if (g_dry) { set_smem(k_px_tma<M, W, ED, PW, PV>, sm); return; }
  static int per_sm = 0;   // resident CTAs per SM (same for every plan)
  if (per_sm == 0) {
    int n = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_px_tma<M, W, ED, PW, PV>, Geo<float, M, W>::NTHR,
                                                     sm));
    per_sm = n > 0 ? n : 1;
  }
  const int64_t nblk = (rows + PG::RG - 1) / PG::RG;
  const int64_t want = ((int64_t)per_sm * g_num_sms_x + count - 1) / count;
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nblk, want));
  ProfScope ps("px", 32, M, s);
  k_px_tma<M, W, ED, PW, PV><<<dim3(gx, (unsigned)count), Geo<float, M, W>::NTHR, sm, s>>>(a);
  g_launches++;
}
template <int M>
void launch_px_tma(const Args& a, int64_t rows, int count, cudaStream_t s) {
  if (g_dry) {
    launch_px_tma_ed<M, false>(a, rows, count, s);
    launch_px_tma_ed<M, true>(a, rows, count, s);
    launch_px_tma_ed<M, false, true>(a, rows, count, s);
    launch_px_tma_ed<M, true, true>(a, rows, count, s);
    launch_px_tma_ed<M, false, false, PV_DYKSTRA>(a, rows, count, s);
    launch_px_tma_ed<M, false, false, PV_ADMM>(a, rows, count, s);
  } else if (a.pv == PV_DYKSTRA) {   // projection variants (lean only)
    launch_px_tma_ed<M, false, false, PV_DYKSTRA>(a, rows, count, s);
  } else if (a.pv == PV_ADMM) {
    launch_px_tma_ed<M, false, false, PV_ADMM>(a, rows, count, s);
  } else if (a.pw_e) {   // pointwise E_n
    if (px_full(a)) launch_px_tma_ed<M, true, true>(a, rows, count, s);
    else launch_px_tma_ed<M, false, true>(a, rows, count, s);
  } else if (px_full(a)) {
    launch_px_tma_ed<M, true>(a, rows, count, s);
  } else {
    launch_px_tma_ed<M, false>(a, rows, count, s);
  }
}

// Persistent bulk-copy-fed entry and exit x passes (float32, one-warp
// tiles), sized like the loop's x pass; K selects the kernel.
template <int M, XKind K, bool PW>
void launch_xio_tma(const Args& a, int64_t rows, int count, cudaStream_t s) {
  constexpr int W = row_w1(M);
  using PG = PxTmaGeo<M, W>;
  const size_t sm = PG::bytes;
  auto kern = K == XFWD ? k_xfwd_tma<M, W, PW> : k_xexit_tma<M, W, PW>;
  if (g_dry) { set_smem(kern, sm); return; }
  static int per_sm = 0;   // resident CTAs per SM (same for every plan)
  if (per_sm == 0) {
    int n = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, Geo<float, M, W>::NTHR, sm));
    per_sm = n > 0 ? n : 1;
  }
  const int64_t nblk = (rows + PG::RG - 1) / PG::RG;
  const int64_t want = ((int64_t)per_sm * g_num_sms_x + count - 1) / count;
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nblk, want));
  ProfScope ps(K == XFWD ? "xfwd" : "xexit", 32, M, s);
  kern<<<dim3(gx, (unsigned)count), Geo<float, M, W>::NTHR, sm, s>>>(a);
  g_launches++;
}
// The entry (measure only: no pre-clip, no mask) and exit (not Dykstra's)
// follow the plan's choice of the persistent x pass.
inline bool xio_tma_ok(XKind kind, const Args& a) {
  if (kind == XFWD) return !(a.mode & (M_PRECLIP | M_MASK));
  return kind == XEXIT && a.pv != PV_DYKSTRA;
}
template <int M, bool PW>
bool launch_xio_tma_kind(XKind kind, const Args& a, int64_t rows, int count, cudaStream_t s) {
  if (g_dry) {   // both bound kinds (the pointwise dry run does not pass w < 0)
    launch_xio_tma<M, XFWD, false>(a, rows, count, s);
    launch_xio_tma<M, XEXIT, false>(a, rows, count, s);
    launch_xio_tma<M, XFWD, true>(a, rows, count, s);
    launch_xio_tma<M, XEXIT, true>(a, rows, count, s);
    return false;
  }
  if (!xio_tma_ok(kind, a)) return false;
  if (kind == XFWD) launch_xio_tma<M, XFWD, PW>(a, rows, count, s);
  else launch_xio_tma<M, XEXIT, PW>(a, rows, count, s);
  return true;
}

template <typename T>
struct XL {
  template <int M>
  static void go(XKind kind, int w, const Args& a, int64_t rows, int count, cudaStream_t s) {
    if (a.pw_e || g_pw_sel) {
      if constexpr (sizeof(T) == 4) {
        // the loop's x passes follow the plan's choice of the copy-engine-fed kernel
        if (w < 0 && kind == XPX && !g_dry) { launch_px_tma<M>(a, rows, count, s); return; }
        if (w < 0 && launch_xio_tma_kind<M, true>(kind, a, rows, count, s)) return;
      }
      launch_x_tw<T, M, row_w1(M), true>(kind, a, rows, count, s);
      return;
    }
    if constexpr (sizeof(T) == 4) {
      // projection variants: the x passes that carry q / u (the loop's pass
      // follows the plan's choice of the persistent kernel)
      if ((a.pv == PV_DYKSTRA || a.pv == PV_ADMM) && kind == XPX && w < 0 && !g_dry) {
        launch_px_tma<M>(a, rows, count, s);
        return;
      }
      if (a.pv == PV_DYKSTRA && (kind == XPX || kind == XEXIT)) {
        launch_x_tw<T, M, row_w1(M), false, PV_DYKSTRA>(kind, a, rows, count, s);
        return;
      }
      if (a.pv == PV_ADMM && kind == XPX) {
        launch_x_tw<T, M, row_w1(M), false, PV_ADMM>(kind, a, rows, count, s);
        return;
      }
    }
    if constexpr (sizeof(T) == 4) {
      if (w < 0 && (kind == XPX || g_dry)) {
        launch_px_tma<M>(a, rows, count, s);
        if (!g_dry) return;
      }
      // the entry and exit passes follow the loop's x-pass choice
      if (w < 0 && launch_xio_tma_kind<M, false>(kind, a, rows, count, s)) return;
      if constexpr (split1_ok<M>()) {
        if ((w & kSplit) && (kind == XPX || g_dry)) {
          if ((w & ~kSplit) == row_w2(M)) launch_x_tw<T, M, row_w2(M), false, PV_POCS, 1>(kind, a, rows, count, s);
          else launch_x_tw<T, M, row_w1(M), false, PV_POCS, 1>(kind, a, rows, count, s);
          if (!g_dry) return;
        }
      }
      if ((w & ~kSplit) == row_w2(M)) launch_x_tw<T, M, row_w2(M)>(kind, a, rows, count, s);
      else launch_x_tw<T, M, row_w1(M)>(kind, a, rows, count, s);
    } else {
      launch_x_tw<T, M, row_w1(M)>(kind, a, rows, count, s);
    }
  }
};
template <typename T>
void launch_x(XKind kind, int M, int w, const Args& a, int64_t rows, int count, cudaStream_t s) {
  FFCZ_DISPATCH_L(M, XL<T>::template go, kind, w, a, rows, count, s)
}

template <typename T, int L, int DIR, int W, int S = 0>
void launch_axis_tw(const Args& a, int Nz, int M, int count, cudaStream_t s) {
  using G_ = Geo<T, L, W>;
  const int64_t tiles = (int64_t)Nz * (M / G_::W);
  dim3 grid((unsigned)((tiles + G_::G - 1) / G_::G), (unsigned)count);
  const size_t sm = Smem<T, L, W>::bytes_axis;
  if (g_dry) { set_smem(k_axis<T, L, DIR, W, S>, sm); return; }
  ProfScope ps(DIR < 0 ? "axis_fwd" : "axis_inv", 8 * (int)sizeof(T), L, s);
  k_axis<T, L, DIR, W, S><<<grid, G_::NTHR, sm, s>>>(a);
  g_launches++;
}
// Persistent TMA-fed variants (float32, 8-pencil tiles, L >= 256): CTAs
// per SM slot and per item as picked at plan time.
int g_num_sms = 148;   // set from the device at plan creation
constexpr int kTmaCtasPerSm = TmaGeo<256, 8>::MINB;   // the kernels' launch bound
inline unsigned tma_grid_x(int64_t tiles, int count) {
  const int64_t want = ((int64_t)kTmaCtasPerSm * g_num_sms + count - 1) / count;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, want));
}
template <int L>
constexpr bool tma_ok() { return Geo<float, L, 8>::G == 1; }

template <int L, int DIR>
void launch_axis_tma(const Args& a, int Nz, int M, int count, cudaStream_t s) {
  const int64_t tiles = (int64_t)Nz * (M / 8);
  const size_t sm = TmaGeo<L, 8>::bytes;
  if (g_dry) { set_smem(k_axis_tma<L, DIR, 8>, sm); return; }
  ProfScope ps(DIR < 0 ? "axis_fwd" : "axis_inv", 32, L, s);
  k_axis_tma<L, DIR, 8><<<dim3(tma_grid_x(tiles, count), (unsigned)count), Geo<float, L, 8>::NTHR, sm, s>>>(a);
  g_launches++;
}
// The check pass needs its full variant for the adjoint's mask modes and for
// edit recording; every other launch takes the lean one.
inline bool chk_full(const Args& a) { return (a.mode & (M_RECORD | M_MASK)) != 0 || a.ed_t != nullptr; }

template <int L>
void launch_chk_tma(const Args& a, int Nmid, int M, int count, cudaStream_t s) {
  const int64_t tiles = chk_ntiles(8, M, Nmid);
  // pointwise bounds or a variant's residual ride in a second staging buffer
  const bool res = a.pv == PV_DYKSTRA || a.pv == PV_DR;
  const size_t sm = (a.pw_f || res) ? TmaGeo<L, 8>::bytes_pw : TmaGeo<L, 8>::bytes;
  if (g_dry) {
    const size_t sp = TmaGeo<L, 8>::bytes_pw;
    set_smem(k_chk_tma<L, 8, true>, TmaGeo<L, 8>::bytes); set_smem(k_chk_tma<L, 8, false>, TmaGeo<L, 8>::bytes);
    set_smem(k_chk_tma<L, 8, true, true>, sp); set_smem(k_chk_tma<L, 8, false, true>, sp);
    set_smem(k_chk_tma<L, 8, false, false, PV_DYKSTRA>, sp); set_smem(k_chk_tma<L, 8, false, false, PV_DR>, sp);
    return;
  }
  ProfScope ps((a.mode & M_NOWRITE) ? "chk_cert" : (a.mode & M_MASK) ? "chk_adj" : "chk", 32, L, s);
  const dim3 grid(tma_grid_x(tiles, count), (unsigned)count);
  const bool full = chk_full(a);
  if (a.pw_f) {   // pointwise (Delta^Re, Delta^Im)
    if (full) k_chk_tma<L, 8, true, true><<<grid, Geo<float, L, 8>::NTHR, sm, s>>>(a);
    else k_chk_tma<L, 8, false, true><<<grid, Geo<float, L, 8>::NTHR, sm, s>>>(a);
  } else if (a.pv == PV_DYKSTRA) {   // the variants run the lean form only
    k_chk_tma<L, 8, false, false, PV_DYKSTRA><<<grid, Geo<float, L, 8>::NTHR, sm, s>>>(a);
  } else if (a.pv == PV_DR) {
    k_chk_tma<L, 8, false, false, PV_DR><<<grid, Geo<float, L, 8>::NTHR, sm, s>>>(a);
  } else if (full) {
    k_chk_tma<L, 8, true><<<grid, Geo<float, L, 8>::NTHR, sm, s>>>(a);
  } else {
    k_chk_tma<L, 8, false><<<grid, Geo<float, L, 8>::NTHR, sm, s>>>(a);
  }
  g_launches++;
}

constexpr int kAxisW64 = 4;   // tile width of the FP64 y pass
template <typename T, int DIR>
struct AL {
  template <int L>
  static void go(int w, const Args& a, int Nz, int M, int count, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
      if constexpr (tma_ok<L>()) {
        if (w < 0 && (a.tm_axis || g_dry)) { launch_axis_tma<L, DIR>(a, Nz, M, count, s); return; }
      }
      if constexpr (split1_ok<L>()) {
        if ((w & kSplit) || g_dry) {
          if ((w & ~kSplit) == 4) launch_axis_tw<T, L, DIR, 4, 1>(a, Nz, M, count, s);
          else launch_axis_tw<T, L, DIR, 8, 1>(a, Nz, M, count, s);
          if (!g_dry) return;
        }
      }
      if ((w & ~kSplit) == 4) launch_axis_tw<T, L, DIR, 4>(a, Nz, M, count, s);
      else launch_axis_tw<T, L, DIR, 8>(a, Nz, M, count, s);
    } else {
      launch_axis_tw<T, L, DIR, kAxisW64>(a, Nz, M, count, s);
    }
  }
};
template <typename T, int DIR>
void launch_axis(int L, int w, const Args& a, int Nz, int M, int count, cudaStream_t s) {
  using D = AL<T, DIR>;
  FFCZ_DISPATCH_L(L, D::template go, w, a, Nz, M, count, s)
}

template <typename T, int L, int W, bool PW = false, int PV = PV_POCS, int S = 0>
void launch_chk_tw(const Args& a, int Nmid, int M, int count, cudaStream_t s) {
  using G_ = Geo<T, L, W>;
  const int64_t tiles = chk_ntiles(W, M, Nmid);
  dim3 grid((unsigned)((tiles + G_::G - 1) / G_::G), (unsigned)count);
  const size_t sm = Smem<T, L, W>::bytes_axis;
  // the full form when a mode needs it; projection variants only run lean
  // (no edits, no adjoint)
  constexpr bool lean_ok = true, only_lean = PV != PV_POCS;
  if (g_dry) {
    if constexpr (!only_lean) set_smem(k_chk<T, L, W, PW, PV, true, S>, sm);
    if constexpr (lean_ok) set_smem(k_chk<T, L, W, PW, PV, false, S>, sm);
    return;
  }
  ProfScope ps((a.mode & M_NOWRITE) ? "chk_cert" : (a.mode & M_MASK) ? "chk_adj" : "chk",
               8 * (int)sizeof(T), L, s);
  if constexpr (lean_ok) {
    if (only_lean || !chk_full(a)) {
      k_chk<T, L, W, PW, PV, false, S><<<grid, G_::NTHR, sm, s>>>(a);
      g_launches++;
      return;
    }
  }
  if constexpr (!only_lean) {
    k_chk<T, L, W, PW, PV, true, S><<<grid, G_::NTHR, sm, s>>>(a);
    g_launches++;
  }
}
template <typename T>
struct CL {
  template <int L>
  static void go(int w, const Args& a, int Nmid, int M, int count, cudaStream_t s) {
    if (a.pw_f || g_pw_sel) {
      if constexpr (sizeof(T) == 4 && tma_ok<L>()) {
        if (w < 0 && a.tm_chk && a.tm_aux && !g_dry) { launch_chk_tma<L>(a, Nmid, M, count, s); return; }
      }
      launch_chk_tw<T, L, TileW<T>::value, true>(a, Nmid, M, count, s);
      return;
    }
    if constexpr (sizeof(T) == 4) {
      // projection variants with a frequency residual (one tile width, or
      // the persistent kernel with the residual staged beside the spectrum)
      if (a.pv == PV_DYKSTRA || a.pv == PV_DR) {
        if constexpr (tma_ok<L>()) {
          if (w < 0 && a.tm_chk && a.tm_aux && !g_dry) { launch_chk_tma<L>(a, Nmid, M, count, s); return; }
        }
        if (a.pv == PV_DYKSTRA) launch_chk_tw<T, L, TileW<T>::value, false, PV_DYKSTRA>(a, Nmid, M, count, s);
        else launch_chk_tw<T, L, TileW<T>::value, false, PV_DR>(a, Nmid, M, count, s);
        return;
      }
    }
    if constexpr (sizeof(T) == 4) {
      if constexpr (tma_ok<L>()) {
        if (w < 0 && (a.tm_chk || g_dry)) { launch_chk_tma<L>(a, Nmid, M, count, s); return; }
      }
      if constexpr (split1_ok<L>()) {
        if ((w & kSplit) || g_dry) {
          if ((w & ~kSplit) == 4) launch_chk_tw<T, L, 4, false, PV_POCS, 1>(a, Nmid, M, count, s);
          else launch_chk_tw<T, L, 8, false, PV_POCS, 1>(a, Nmid, M, count, s);
          if (!g_dry) return;
        }
      }
      if ((w & ~kSplit) == 4) launch_chk_tw<T, L, 4>(a, Nmid, M, count, s);
      else launch_chk_tw<T, L, 8>(a, Nmid, M, count, s);
    } else {
      launch_chk_tw<T, L, 4>(a, Nmid, M, count, s);
    }
  }
};
template <typename T>
void launch_chk(int L, int w, const Args& a, int Nmid, int M, int count, cudaStream_t s) {
  FFCZ_DISPATCH_L(L, CL<T>::template go, w, a, Nmid, M, count, s)
}

// ----- 1D (Bluestein) passes ---------------------------------------------------
template <typename T, int L, int W>
void launch_col1_tw(const Args& a, int P2, int count, cudaStream_t s) {
  using G_ = Geo<T, L, W>;
  const int64_t tiles = P2 / G_::W;
  dim3 grid((unsigned)((tiles + G_::G - 1) / G_::G), (unsigned)count);
  const size_t sm = Smem<T, L, W>::bytes_axis;
  if (g_dry) { set_smem(k1_col<T, L, W>, sm); return; }
  ProfScope ps(a.op1 == OP1_FCLIP ? ((a.mode & M_NOWRITE) ? "col1_cert" : "col1_fclip")
               : a.op1 == OP1_SCLIP ? "col1_sclip" : a.op1 == OP1_EXIT ? "col1_exit"
               : a.op1 == OP1_FILTER ? "col1_filter" : a.op1 == OP1_ZOUT ? "col1_zout" : "col1_entry",
               8 * (int)sizeof(T), L, s);
  k1_col<T, L, W><<<grid, G_::NTHR, sm, s>>>(a);
  g_launches++;
}
template <typename T>
struct C1L {
  template <int L>
  static void go(int w, const Args& a, int P2, int count, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
      if (w == 4) launch_col1_tw<T, L, 4>(a, P2, count, s);
      else launch_col1_tw<T, L, 8>(a, P2, count, s);
    } else {
      launch_col1_tw<T, L, 4>(a, P2, count, s);
    }
  }
};
template <typename T>
void launch_col1(int L, int w, const Args& a, int P2, int count, cudaStream_t s) {
  FFCZ_DISPATCH_L(L, C1L<T>::template go, w, a, P2, count, s)
}
template <typename T, int L, int W>
void launch_row1_tw(const Args& a, int P1, int count, cudaStream_t s) {
  using G_ = Geo<T, L, W>;
  const int64_t tiles = (P1 + G_::W - 1) / G_::W;
  dim3 grid((unsigned)((tiles + G_::G - 1) / G_::G), (unsigned)count);
  const size_t sm = Smem<T, L, W>::bytes_axis;
  if (g_dry) { set_smem(k1_row<T, L, W>, sm); return; }
  ProfScope ps(a.op1 == OP1_FWD ? "row1_fwd" : "row1_conv", 8 * (int)sizeof(T), L, s);
  k1_row<T, L, W><<<grid, G_::NTHR, sm, s>>>(a);
  g_launches++;
}
template <typename T>
struct R1L {
  template <int L>
  static void go(int w, const Args& a, int P1, int count, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
      if (w == row_w2(L)) launch_row1_tw<T, L, row_w2(L)>(a, P1, count, s);
      else launch_row1_tw<T, L, row_w1(L)>(a, P1, count, s);
    } else {
      launch_row1_tw<T, L, row_w1(L)>(a, P1, count, s);
    }
  }
};
template <typename T>
void launch_row1(int L, int w, const Args& a, int P1, int count, cudaStream_t s) {
  FFCZ_DISPATCH_L(L, R1L<T>::template go, w, a, P1, count, s)
}

// Words of mask storage one float32 pass writes: MW words per thread of
// every tile (tiles x threads per tile x words per thread).
inline int64_t mask_words_per_thread(int L) { return (f2_v(L) + 7) / 8; }
// Tile width of a tuner width code (fft_core.cuh split flag and the
// persistent kernel's sign removed).
inline int code_width(int w) { return std::abs(w) & ~kSplit; }
inline int64_t x_words(int M, int64_t rows, int W) {
  W = code_width(W);
  const int64_t tiles = (rows + W - 1) / W;
  return tiles * (int64_t)f2_nt(M) * W * mask_words_per_thread(M);
}
inline int64_t chkw(int L, int Nmid, int M, int W) {
  W = code_width(W);   // the TMA-fed variant (-8) tiles like the 8-pencil one
  return (int64_t)chk_ntiles(W, M, Nmid) * f2_nt(L) * W * mask_words_per_thread(L);
}

// ----- argument construction ------------------------------------------------
int cnt_flag(const ffcz_plan_s* p) { return p->opts.count_active ? M_COUNT : 0; }

// ----- TMA tensor maps ------------------------------------------------------
// The encoder is the driver's cuTensorMapEncodeTiled, reached through the
// runtime's entry-point query (no link against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    (void)cudaGetLastError();
  });
  return fn;
}

// 2D view [outer][inner] of 8-byte elements (one complex64 each) at base,
// row pitch inner * 8 bytes, boxes of boxw x boxr elements.
bool encode_2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint32_t boxw,
               uint32_t boxr) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15u) || (inner * 8) % 16 || inner < boxw || outer < boxr) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 8};
  cuuint32_t box[2] = {boxw, boxr};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Maps of both float32 spectrum buffers for every member of every 2D/3D
// group: the y pass reads tiles of the [Nz Ny][M] view, the check pass of
// the [Nz][Nmid M] view, in boxes of 8 pencils x min(L, 256) rows.  The
// TMA-fed kernels exist for pencil lengths L >= 256 (tiles of one CTA).
void build_tensor_maps(ffcz_plan_s* p) {
  for (auto& dg : p->groups) {
    if (dg.ndim == 1) continue;
    const int Nmid = dg.ndim == 3 ? dg.Ny : 1;
    for (int kind = 0; kind < 2; ++kind) {
      if (kind == 0 && dg.ndim != 3) continue;
      const int L = kind == 0 ? dg.Ny : dg.Nz;
      if (L < 256) continue;
      std::vector<CUtensorMap> maps(2 * (size_t)dg.count);
      bool ok = true;
      for (int gi = 0; gi < dg.count && ok; ++gi)
        for (int b = 0; b < 2 && ok; ++b) {
          const char* base = static_cast<const char*>(p->B32[b]) + dg.h_soff[gi] * 8;
          const uint32_t rows = (uint32_t)std::min(L, 256);
          ok = kind == 0 ? encode_2d(&maps[2 * gi + b], base, (uint64_t)dg.M, (uint64_t)dg.Nz * dg.Ny, 8, rows)
                         : encode_2d(&maps[2 * gi + b], base, (uint64_t)Nmid * dg.M, (uint64_t)dg.Nz, 8, rows);
        }
      if (!ok) continue;
      void* d = dalloc(p, sizeof(CUtensorMap) * maps.size());
      CK(cudaMemcpy(d, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice));
      (kind == 0 ? dg.tm_axis : dg.tm_chk) = static_cast<const CUtensorMap*>(d);
    }
  }
}

// The check pass's [Nz][Nmid M] view of an auxiliary packed field (the
// pointwise f-bounds, or the Dykstra / Douglas-Rachford residual) of every
// member (same boxes as the spectrum maps), where that pass has a TMA-fed
// kernel.
void build_aux_maps(ffcz_plan_s* p, const void* field) {
  for (auto& dg : p->groups) {
    if (dg.ndim == 1 || !dg.tm_chk) continue;
    const int Nmid = dg.ndim == 3 ? dg.Ny : 1;
    std::vector<CUtensorMap> maps((size_t)dg.count);
    bool ok = true;
    for (int gi = 0; gi < dg.count && ok; ++gi) {
      const char* base = static_cast<const char*>(field) + dg.h_soff[gi] * 8;
      ok = encode_2d(&maps[gi], base, (uint64_t)Nmid * dg.M, (uint64_t)dg.Nz, 8, (uint32_t)std::min(dg.Nz, 256));
    }
    if (!ok) continue;
    void* d = dalloc(p, sizeof(CUtensorMap) * maps.size());
    CK(cudaMemcpy(d, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice));
    dg.tm_aux = static_cast<const CUtensorMap*>(d);
  }
}

template <typename T>
Args make_args(ffcz_plan_s* p, const DevGroup& dg, void* b0, void* b1, ItemState* st) {
  Args a{};
  a.g = dg.g;
  a.prm = p->d_prm;
  a.st = st;
  a.B0 = b0;
  a.B1 = b1;
  a.pred = P_ACTIVE;
  a.sel_in = a.sel_out = S_CUR;
  a.ckpt_every = 0;
  a.ckpt_stride = p->total;
  a.mask_thr = 0;
  a.err = p->d_err;
  if (p->opts.pointwise) {
    a.pw_e = p->pw_e;
    a.pw_f = p->ndim == 1 ? p->pw_f : p->pw_fp;   // 1D: bins k <= N/2 of each item
    a.pw_f0 = p->pw_f0;
  }
  if (p->ed_on) {
    a.ed_s = p->ed_s;
    a.ed_f = p->ed_f;
    a.ed_p = p->ed_p;
    a.ed_t = p->ed_t;
  }
  if (sizeof(T) == 4 && b0 == p->B32[0] && b1 == p->B32[1]) {
    a.tm_axis = dg.tm_axis;
    a.tm_chk = dg.tm_chk;
    a.tm_aux = dg.tm_aux;
  }
  if (sizeof(T) == 4 && p->pv_on) {
    a.pv = p->opts.method;
    a.pv_r = p->pv_r;
    a.pv_q[0] = p->pv_q[0];
    a.pv_q[1] = p->pv_q[1];
  }
  return a;
}

template <typename T>
void tabs_x(ffcz_plan_s* p, Args& a, const DevGroup& dg) {
  set_tw<T>(a, p->tb, dg.M);
  a.twr = twr_of<T>(p->tb, dg.Nx);
}

template <typename T>
void col1_args(ffcz_plan_s* p, Args& a, const DevGroup& dg, int op) {
  set_tw<T>(a, p->tb, dg.P1);
  a.twr = sizeof(T) == 4 ? dg.twp32 : dg.twp64;
  a.chirp = sizeof(T) == 4 ? p->ch32 : p->ch64;
  a.op1 = op;
}
template <typename T>
void row1_args(ffcz_plan_s* p, Args& a, const DevGroup& dg, int op) {
  set_tw<T>(a, p->tb, dg.P2);
  a.bt = sizeof(T) == 4 ? p->Bt32 : p->Bt64;
  a.op1 = op;
}

// ----- multi-group form of the loop passes -------------------------------------
// The pass length and the two extents (multi_grid_of) of kind k for group dg.
int multi_len(int k, const DevGroup& dg) {
  switch (k) {
    case MK_PX: return dg.M;
    case MK_YINV: case MK_YFWD: return dg.Ny;
    case MK_CHK: return dg.Nz;
    case MK_COL1: return dg.P1;
    default: return dg.P2;
  }
}
template <int KIND>
struct MG {
  template <int L>
  static void go(const DevGroup& dg, MultiGrid& r) {
    if constexpr (KIND == MK_PX) r = multi_grid_of<KIND, L>(dg.rows, 0);
    else if constexpr (KIND == MK_YINV || KIND == MK_YFWD) r = multi_grid_of<KIND, L>(dg.Nz, dg.M);
    else if constexpr (KIND == MK_CHK) r = multi_grid_of<KIND, L>(dg.M, dg.ndim == 3 ? dg.Ny : 1);
    else if constexpr (KIND == MK_COL1) r = multi_grid_of<KIND, L>(dg.P2, 0);
    else r = multi_grid_of<KIND, L>(dg.P1, 0);
  }
};
template <int KIND>
MultiGrid multi_grid(const DevGroup& dg) {
  MultiGrid r{0, 0};
  FFCZ_DISPATCH_L(multi_len(KIND, dg), MG<KIND>::template go, dg, r)
  return r;
}
template <int KIND>
void* multi_kernel() { return reinterpret_cast<void*>(&k_multi<KIND>); }

// Work list of kind KIND over every group (groups of longer transforms
// first, then member by member), its shared memory and the grid of its
// persistent launch (as many 128-thread CTAs as fit on the device).
template <int KIND>
void build_multi_kind(ffcz_plan_s* p) {
  const int ng = (int)p->groups.size();
  std::vector<int> order(ng);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return multi_len(KIND, p->groups[x]) > multi_len(KIND, p->groups[y]);
  });
  std::vector<int2> units;
  size_t smem = 0;
  for (int g : order) {
    const DevGroup& dg = p->groups[g];
    const MultiGrid mg = multi_grid<KIND>(dg);
    smem = std::max(smem, mg.smem);
    for (int gi = 0; gi < dg.count; ++gi)
      for (int64_t bx = 0; bx < mg.gx; ++bx) units.push_back(make_int2(g | (gi << 4), (int)bx));
  }
  auto& m = p->mp[KIND];
  m.n = (int64_t)units.size();
  m.smem = smem;
  if (smem > 48 * 1024)
    CK(cudaFuncSetAttribute(k_multi<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi<KIND>, kMultiThreads, smem));
  m.grid = (int)std::min<int64_t>(m.n, (int64_t)std::max(per_sm, 1) * p->num_sms);
  m.units = static_cast<int2*>(dalloc(p, sizeof(int2) * units.size()));
  CK(cudaMemcpy(m.units, units.data(), sizeof(int2) * units.size(), cudaMemcpyHostToDevice));
}

// Work lists of the pass kinds the plan's loop runs, for plans of 2 to
// kMultiGroups groups.
void build_multi(ffcz_plan_s* p) {
  const int ng = (int)p->groups.size();
  if (ng < 2 || ng > kMultiGroups) return;
  if (p->ndim == 1) {
    build_multi_kind<MK_COL1>(p);
    build_multi_kind<MK_ROW1>(p);
    return;
  }
  build_multi_kind<MK_PX>(p);
  build_multi_kind<MK_CHK>(p);
  if (p->ndim == 3) {
    build_multi_kind<MK_YINV>(p);
    build_multi_kind<MK_YFWD>(p);
  }
}

const char* multi_name(int k) {
  static const char* n[MK_N] = {"px", "axis_inv", "axis_fwd", "chk", "col1", "row1"};
  return n[k];
}
// profile key of a multi-group launch ("multi_chk<f32,0>": every length)
const char* multi_prof_name(int k) {
  static const char* n[MK_N] = {"multi_px", "multi_axis_inv", "multi_axis_fwd", "multi_chk", "multi_col1",
                                "multi_row1"};
  return n[k];
}
void* multi_kernel_of(int k) {
  switch (k) {
    case MK_PX: return multi_kernel<MK_PX>();
    case MK_YINV: return multi_kernel<MK_YINV>();
    case MK_YFWD: return multi_kernel<MK_YFWD>();
    case MK_CHK: return multi_kernel<MK_CHK>();
    case MK_COL1: return multi_kernel<MK_COL1>();
    default: return multi_kernel<MK_ROW1>();
  }
}

// One multi-group launch of kind k with the per-group arguments `args`
// (p->groups order), if the plan took the multi-group form for k and every
// argument set is one the form covers (float32, Alg. 1, no pointwise
// bounds, lean passes: no adjoint modes, checkpoints or edit recording).
// Returns false if the caller must launch the groups separately.
template <typename T>
bool multi_launch(ffcz_plan_s* p, int k, const std::vector<Args>& args, cudaStream_t s, bool force = false) {
  if constexpr (sizeof(T) != 4) {
    return false;
  } else {
    const auto& m = p->mp[k];
    if ((!p->multi_use[k] && !force) || m.n == 0 || g_pw_sel) return false;
    for (size_t g = 0; g < args.size(); ++g) {
      const Args& a = args[g];
      if (a.pw_e || a.pw_f || a.pv != PV_POCS) return false;
      // the multi-group units run the default radix split
      const DevGroup& dg = p->groups[g];
      const int w = k == MK_PX ? dg.wx : (k == MK_YINV || k == MK_YFWD) ? dg.wa : k == MK_CHK ? dg.wc : 0;
      if (w > 0 && (w & kSplit)) return false;
      if (k == MK_PX && px_full(a)) return false;
      if (k == MK_CHK && chk_full(a)) return false;
    }
    MultiArgs ma{};
    for (size_t g = 0; g < args.size(); ++g) {
      ma.a[g] = args[g];
      ma.len[g] = multi_len(k, p->groups[g]);
    }
    ma.units = m.units;
    ma.nunits = m.n;
    ProfScope ps(multi_prof_name(k), 32, 0, s);
    void* params[] = {&ma};
    CK(cudaLaunchKernel(multi_kernel_of(k), dim3((unsigned)m.grid), dim3(kMultiThreads), params, m.smem, s));
    g_launches++;
    return true;
  }
}

// Chirp tables and Bt = FFT_P(wrapped chirp) for every 1D item, in the
// precision T.
template <typename T>
void build_bt(ffcz_plan_s* p) {
  void*& ch = sizeof(T) == 4 ? p->ch32 : p->ch64;
  if (!ch) ch = dalloc(p, (size_t)p->total * sizeof(v2<T>));
  for (auto& dg : p->groups) {
    dim3 grid(64, (unsigned)dg.count);
    k1_chirp_table<T><<<grid, 256, 0, p->stream>>>(dg.g, p->d_prm, reinterpret_cast<v2<T>*>(ch));
    g_launches++;
  }
  void*& bt = sizeof(T) == 4 ? p->Bt32 : p->Bt64;
  if (!bt) bt = dalloc(p, (size_t)p->total_c * sizeof(v2<T>));
  for (auto& dg : p->groups) {
    Args a = make_args<T>(p, dg, bt, bt, p->d_st);
    a.pred = P_ALL;
    col1_args<T>(p, a, dg, OP1_FILTER);
    launch_col1<T>(dg.P1, dg.w1c, a, dg.P2, dg.count, p->stream);
    row1_args<T>(p, a, dg, OP1_FWD);
    launch_row1<T>(dg.P2, dg.w1r, a, dg.P1, dg.count, p->stream);
  }
}

// ----- the loop ---------------------------------------------------------------
// 1 when the loop's stopping test is ADMM's spatial check (k_decide)
template <typename T>
int s_check_of(const ffcz_plan_s* p) {
  return (sizeof(T) == 4 && p->pv_on && p->opts.method == PV_ADMM) ? 1 : 0;
}

struct LoopBufs {
  void* b0;
  void* b1;
};

// The differentiable forward keeps every step's masks (float32 loops).
template <typename T>
bool keep_masks_rec(const ffcz_plan_s* p) {
  return sizeof(T) == 4 && p->ck_rec && p->opts.keep_masks && p->km_s;
}
int64_t px_mask_thr(const DevGroup& dg);
int64_t chk_mask_thr(const DevGroup& dg);
// x pass (s-masks) or check pass (f-masks) of group g records into the
// plan's per-step mask store
void km_args(ffcz_plan_s* p, Args& a, int g, bool chk) {
  const DevGroup& dg = p->groups[g];
  a.mode |= M_RECORD;
  if (p->ndim == 1) {   // mask bytes at the items' point offsets
    a.mask = chk ? p->km_f : p->km_s;
    a.mask_step = chk ? p->chk_words : p->px_words;
    return;
  }
  a.mask = chk ? p->km_f + p->bw_chkoff[g] : p->km_s + p->bw_pxoff[g];
  a.mask_thr = chk ? chk_mask_thr(dg) : px_mask_thr(dg);
  a.mask_step = chk ? p->chk_words : p->px_words;
}

template <typename T>
void entry1(ffcz_plan_s* p, LoopBufs B, float* e, bool measure_preclip, cudaStream_t s) {
  for (auto& dg : p->groups) {
    Args a = make_args<T>(p, dg, B.b0, B.b1, p->d_st);
    col1_args<T>(p, a, dg, OP1_ENTRY);
    a.e = e;
    a.mode = measure_preclip ? M_MEASURE : 0;
    launch_col1<T>(dg.P1, dg.w1c, a, dg.P2, dg.count, s);
  }
  if (measure_preclip) {
    k_mark_preclip<<<(unsigned)((p->batch + 255) / 256), 256, 0, s>>>(p->d_prm, p->d_st, (int)p->batch);
    g_launches++;
    for (auto& dg : p->groups) {
      Args a = make_args<T>(p, dg, B.b0, B.b1, p->d_st);
      col1_args<T>(p, a, dg, OP1_ENTRY);
      a.e = e;
      a.mode = M_PRECLIP;
      a.pred = P_PRECLIP;
      launch_col1<T>(dg.P1, dg.w1c, a, dg.P2, dg.count, s);
    }
  }
  for (auto& dg : p->groups) {
    Args a = make_args<T>(p, dg, B.b0, B.b1, p->d_st);
    row1_args<T>(p, a, dg, OP1_CONV);
    launch_row1<T>(dg.P2, dg.w1r, a, dg.P1, dg.count, s);
    col1_args<T>(p, a, dg, OP1_FCLIP);
    a.mode = M_CLIP | cnt_flag(p);
    if (keep_masks_rec<T>(p)) km_args(p, a, 0, true);
    launch_col1<T>(dg.P1, dg.w1c, a, dg.P2, dg.count, s);
  }
  k_decide<<<(unsigned)((p->batch + 255) / 256), 256, 0, s>>>(p->d_prm, p->d_st, (int)p->batch,
                                                             p->d_nactive);
  g_launches++;
}

template <typename T>
void body1(ffcz_plan_s* p, LoopBufs B, cudaStream_t s) {
  // four passes, each over every group (one launch per group, or one
  // multi-group launch); items of different groups are independent, so
  // only the order of the passes matters
  const int ng = (int)p->groups.size();
  std::vector<Args> args(ng);
  for (int step = 0; step < 4; ++step) {
    const bool row = step % 2 == 0;
    for (int g = 0; g < ng; ++g) {
      const DevGroup& dg = p->groups[g];
      Args a = make_args<T>(p, dg, B.b0, B.b1, p->d_st);
      a.sel_in = a.sel_out = S_CUR;
      if (step == 0) { row1_args<T>(p, a, dg, OP1_CONVC); a.sel_in = S_PREV; }
      if (step == 1) {
        col1_args<T>(p, a, dg, OP1_SCLIP);
        a.mode = M_CLIP | cnt_flag(p);
        if (sizeof(T) == 4 && p->ck_rec) {   // the differentiable forward's checkpoints
          a.mode |= M_CKPT;
          a.ckpt = p->bw_ck;
          a.ckpt_every = p->bw_m;
        }
        if (keep_masks_rec<T>(p)) km_args(p, a, g, false);
      }
      if (step == 2) { row1_args<T>(p, a, dg, OP1_CONV); a.mode = 0; }
      if (step == 3) {
        col1_args<T>(p, a, dg, OP1_FCLIP);
        a.mode = M_CLIP | cnt_flag(p);
        if (keep_masks_rec<T>(p)) km_args(p, a, g, true);
      }
      args[g] = a;
    }
    if (multi_launch<T>(p, row ? MK_ROW1 : MK_COL1, args, s)) continue;
    for (int g = 0; g < ng; ++g) {
      const DevGroup& dg = p->groups[g];
      if (row) launch_row1<T>(dg.P2, dg.w1r, args[g], dg.P1, dg.count, s);
      else launch_col1<T>(dg.P1, dg.w1c, args[g], dg.P2, dg.count, s);
    }
  }
  k_decide<<<(unsigned)((p->batch + 255) / 256), 256, 0, s>>>(p->d_prm, p->d_st, (int)p->batch,
                                                             p->d_nactive, s_check_of<T>(p));
  g_launches++;
}

template <typename T>
void exit1(ffcz_plan_s* p, LoopBufs B, float* e, cudaStream_t s) {
  for (auto& dg : p->groups) {
    Args a = make_args<T>(p, dg, B.b0, B.b1, p->d_st);
    a.pred = P_EXIT;
    a.e = e;
    row1_args<T>(p, a, dg, OP1_CONVC);
    a.sel_in = S_PREV; a.sel_out = S_CUR;
    launch_row1<T>(dg.P2, dg.w1r, a, dg.P1, dg.count, s);
    a.sel_in = S_CUR;
    col1_args<T>(p, a, dg, OP1_EXIT);
    // ADMM returns a_t, which its check found inside the s-cube, unclipped
    a.mode = s_check_of<T>(p) ? 0 : M_CLIP;
    launch_col1<T>(dg.P1, dg.w1c, a, dg.P2, dg.count, s);
  }
}

template <typename T>
void entry(ffcz_plan_s* p, LoopBufs B, float* e, bool measure_preclip, cudaStream_t s) {
  if (p->ndim == 1) { entry1<T>(p, B, e, measure_preclip, s); return; }
  for (auto& dg : p->groups) {
    Args a = make_args<T>(p, dg, B.b0, B.b1, p->d_st);
    tabs_x<T>(p, a, dg);
    a.e = e;
    a.mode = measure_preclip ? M_MEASURE : 0;
    launch_x<T>(XFWD, dg.M, dg.wx, a, dg.rows, dg.count, s);
  }
  if (measure_preclip) {
    k_mark_preclip<<<(unsigned)((p->batch + 255) / 256), 256, 0, s>>>(p->d_prm, p->d_st, (int)p->batch);
    g_launches++;
    for (auto& dg : p->groups) {
      Args a = make_args<T>(p, dg, B.b0, B.b1, p->d_st);
      tabs_x<T>(p, a, dg);
      a.e = e;
      a.mode = M_PRECLIP;
      a.pred = P_PRECLIP;
      launch_x<T>(XFWD, dg.M, dg.wx, a, dg.rows, dg.count, s);
    }
  }
  for (size_t g = 0; g < p->groups.size(); ++g) {
    const DevGroup& dg = p->groups[g];
    Args a = make_args<T>(p, dg, B.b0, B.b1, p->d_st);
    if (dg.ndim == 3) {
      set_tw<T>(a, p->tb, dg.Ny);
      launch_axis<T, -1>(dg.Ny, dg.wa, a, dg.Nz, dg.M, dg.count, s);
    }
    set_tw<T>(a, p->tb, dg.Nz);
    a.mode = M_CLIP | cnt_flag(p);
    if (keep_masks_rec<T>(p)) km_args(p, a, (int)g, true);
    launch_chk<T>(dg.Nz, dg.wc, a, dg.ndim == 3 ? dg.Ny : 1, dg.M, dg.count, s);
  }
  k_decide<<<(unsigned)((p->batch + 255) / 256), 256, 0, s>>>(p->d_prm, p->d_st, (int)p->batch,
                                                             p->d_nactive, s_check_of<T>(p));
  g_launches++;
}

template <typename T>
void body(ffcz_plan_s* p, LoopBufs B, cudaStream_t s) {
  if (p->ndim == 1) { body1<T>(p, B, s); return; }
  // y inverse (3D), x pass, y forward (3D), check pass, each over every
  // group (one launch per group, or one multi-group launch); items of
  // different groups are independent, so only the order of the passes matters
  const int ng = (int)p->groups.size();
  const bool three = p->ndim == 3;
  std::vector<Args> args(ng);
  if (three) {
    for (int g = 0; g < ng; ++g) {
      const DevGroup& dg = p->groups[g];
      Args a = make_args<T>(p, dg, B.b0, B.b1, p->d_st);
      set_tw<T>(a, p->tb, dg.Ny);
      a.sel_in = S_PREV; a.sel_out = S_CUR;
      args[g] = a;
    }
    if (!multi_launch<T>(p, MK_YINV, args, s))
      for (int g = 0; g < ng; ++g) {
        const DevGroup& dg = p->groups[g];
        launch_axis<T, +1>(dg.Ny, dg.wa, args[g], dg.Nz, dg.M, dg.count, s);
      }
  }
  for (int g = 0; g < ng; ++g) {
    const DevGroup& dg = p->groups[g];
    Args a = make_args<T>(p, dg, B.b0, B.b1, p->d_st);
    a.sel_in = three ? S_CUR : S_PREV;
    a.sel_out = S_CUR;
    tabs_x<T>(p, a, dg);
    a.mode = M_CLIP | cnt_flag(p);
    if (sizeof(T) == 4 && p->ck_rec) {
      a.mode |= M_CKPT;
      a.ckpt = p->bw_ck;
      a.ckpt_every = p->bw_m;
    }
    if (keep_masks_rec<T>(p)) km_args(p, a, g, false);
    args[g] = a;
  }
  if (!multi_launch<T>(p, MK_PX, args, s))
    for (int g = 0; g < ng; ++g) {
      const DevGroup& dg = p->groups[g];
      launch_x<T>(XPX, dg.M, dg.wx, args[g], dg.rows, dg.count, s);
    }
  if (three) {
    for (int g = 0; g < ng; ++g) {
      const DevGroup& dg = p->groups[g];
      Args a = make_args<T>(p, dg, B.b0, B.b1, p->d_st);
      a.sel_in = a.sel_out = S_CUR;
      set_tw<T>(a, p->tb, dg.Ny);
      a.mode = 0;
      args[g] = a;
    }
    if (!multi_launch<T>(p, MK_YFWD, args, s))
      for (int g = 0; g < ng; ++g) {
        const DevGroup& dg = p->groups[g];
        launch_axis<T, -1>(dg.Ny, dg.wa, args[g], dg.Nz, dg.M, dg.count, s);
      }
  }
  for (int g = 0; g < ng; ++g) {
    const DevGroup& dg = p->groups[g];
    Args a = make_args<T>(p, dg, B.b0, B.b1, p->d_st);
    a.sel_in = a.sel_out = S_CUR;
    set_tw<T>(a, p->tb, dg.Nz);
    a.mode = M_CLIP | cnt_flag(p);
    if (keep_masks_rec<T>(p)) km_args(p, a, g, true);
    args[g] = a;
  }
  if (!multi_launch<T>(p, MK_CHK, args, s))
    for (int g = 0; g < ng; ++g) {
      const DevGroup& dg = p->groups[g];
      launch_chk<T>(dg.Nz, dg.wc, args[g], dg.ndim == 3 ? dg.Ny : 1, dg.M, dg.count, s);
    }
  k_decide<<<(unsigned)((p->batch + 255) / 256), 256, 0, s>>>(p->d_prm, p->d_st, (int)p->batch,
                                                             p->d_nactive, s_check_of<T>(p));
  g_launches++;
}

template <typename T>
void exit_pass(ffcz_plan_s* p, LoopBufs B, float* e, cudaStream_t s) {
  if (p->ndim == 1) { exit1<T>(p, B, e, s); return; }
  for (auto& dg : p->groups) {
    Args a = make_args<T>(p, dg, B.b0, B.b1, p->d_st);
    a.pred = P_EXIT;
    a.e = e;
    if (dg.ndim == 3) {
      set_tw<T>(a, p->tb, dg.Ny);
      a.sel_in = S_PREV; a.sel_out = S_CUR;
      launch_axis<T, +1>(dg.Ny, dg.wa, a, dg.Nz, dg.M, dg.count, s);
      a.sel_in = S_CUR;
    } else {
      a.sel_in = S_PREV;
    }
    tabs_x<T>(p, a, dg);
    // ADMM returns a_t, which its check found inside the s-cube, unclipped
    a.mode = s_check_of<T>(p) ? 0 : M_CLIP;
    launch_x<T>(XEXIT, dg.M, dg.wx, a, dg.rows, dg.count, s);
  }
}

template <typename T>
LoopBufs loop_bufs(ffcz_plan_s* p) {
  // 1D plans need the chirp spectrum in the loop's precision
  if (p->ndim == 1 && sizeof(T) == 8 && !p->Bt64) build_bt<double>(p);
  if (sizeof(T) == 4) return {p->B32[0], p->B32[1]};
  if (!p->B64[0]) {
    p->B64[0] = dalloc(p, (size_t)p->total_c * sizeof(double2));
    p->B64[1] = dalloc(p, (size_t)p->total_c * sizeof(double2));
  }
  return {p->B64[0], p->B64[1]};
}

// Loop control inside a graph: counts executed bodies and keeps the WHILE
// node running while some item is active and the cap is not reached.
__global__ void k_loop_ctl(cudaGraphConditionalHandle h, const int* n_active, int* count, int cap) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int c = *count + 1;
  *count = c;
  cudaGraphSetConditional(h, (*n_active > 0 && c < cap) ? 1u : 0u);
}

// Whole loop on the device: a graph with one conditional WHILE node whose
// body is one captured iteration followed by k_loop_ctl (built once per plan
// and precision, replayed by one cudaGraphLaunch per call).
template <typename T>
void run_while_graph(ffcz_plan_s* p, LoopBufs B, int cap) {
  const int ckk = ((sizeof(T) == 4 && p->ck_rec) ? 1 : 0) + (keep_masks_rec<T>(p) ? 2 : 0);
  const auto key = std::make_pair(-(int)sizeof(T), ckk);
  auto it = p->graphs.find(key);
  if (it == p->graphs.end()) {
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
    cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
    const int64_t before = g_launches.load();
    CK(cudaStreamBeginCaptureToGraph(p->cap_stream, bodyg, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    try {
      body<T>(p, B, p->cap_stream);
      k_loop_ctl<<<1, 32, 0, p->cap_stream>>>(h, p->d_nactive, p->d_loopcount, cap);
    } catch (...) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(p->cap_stream, &junk);
      cudaGraphDestroy(g);
      throw;
    }
    cudaGraph_t captured = nullptr;
    CK(cudaStreamEndCapture(p->cap_stream, &captured));
    const int per_body = (int)(g_launches.load() - before) + 1;
    g_launches -= (g_launches.load() - before);
    cudaGraphExec_t ge;
    CK(cudaGraphInstantiate(&ge, g, 0));
    cudaGraphDestroy(g);
    it = p->graphs.emplace(key, ge).first;
    p->graph_nodes[key] = per_body;
    p->while_cap[sizeof(T) == 4 ? 0 : 1][ckk] = cap;
  }
  CK(cudaMemsetAsync(p->d_loopcount, 0, sizeof(int), p->stream));
  CK(cudaGraphLaunch(it->second, p->stream));
  // kernels per executed body; the count read back with the stats
  p->pending_bodies_per = p->graph_nodes[key];
}

template <typename T>
void run_chunk(ffcz_plan_s* p, LoopBufs B, int C) {
  if (!p->opts.use_graph || p->prof) {
    for (int i = 0; i < C; ++i) body<T>(p, B, p->stream);
    return;
  }
  const auto key = std::make_pair((int)sizeof(T) + ((sizeof(T) == 4 && p->ck_rec) ? 16 : 0) +
                                      (keep_masks_rec<T>(p) ? 32 : 0), C);
  auto it = p->graphs.find(key);
  if (it == p->graphs.end()) {
    cudaGraph_t g;
    const int64_t before = g_launches.load();
    CK(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    try {
      for (int i = 0; i < C; ++i) body<T>(p, B, p->cap_stream);
    } catch (...) {
      cudaGraph_t junk;
      cudaStreamEndCapture(p->cap_stream, &junk);
      if (junk) cudaGraphDestroy(junk);
      throw;
    }
    CK(cudaStreamEndCapture(p->cap_stream, &g));
    g_launches -= (g_launches.load() - before);   // captured, not launched
    cudaGraphExec_t ge;
    CK(cudaGraphInstantiate(&ge, g, 0));
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    cudaGraphDestroy(g);
    it = p->graphs.emplace(key, ge).first;
    p->graph_nodes[key] = (int)nn;
  }
  CK(cudaGraphLaunch(it->second, p->stream));
  g_launches += p->graph_nodes[key];
}

// Bluestein length of a 1D item: the smallest power of two >= 2N - 1.
int64_t p1d_len(int64_t n) {
  int64_t P = 64;
  while (P < 2 * n - 1) P <<= 1;
  return P;
}
// 1D items certified through the N/2-point transform: even N >= 64 (then
// the N/2-point Bluestein length is P/2 >= 64).
inline bool half_cert_ok(int64_t n) { return n % 2 == 0 && n >= 64; }

void upload_params(ffcz_plan_s* p, const double* eps_s, const double* eps_f, int min_iters,
                   int max_iters) {
  const double eta = p->opts.shrink;
  for (int64_t i = 0; i < p->batch; ++i) {
    ItemParams& q = p->h_prm[i];
    const double E = eps_s[i], D = eps_f[i];
    if (!(E > 0) || !(D > 0) || !std::isfinite(E) || !std::isfinite(D))
      fail(FFCZ_ERR_INVALID, "bounds must be finite and > 0");
    int64_t n = 1;
    for (int d = 0; d < p->ndim; ++d) n *= p->shapes[i * p->ndim + d];
    q.E = E; q.D = D;
    q.Es = E * (1.0 - eta); q.Ds = D * (1.0 - eta); q.thr = D * (1.0 - eta / 2.0);
    q.inv_n = 1.0 / (double)n;
    q.Esf = (float)q.Es; q.Dsf = (float)q.Ds; q.thrf = (float)q.thr; q.inv_nf = (float)q.inv_n;
    q.n = n;
    q.min_iters = min_iters;
    q.max_iters = max_iters;
    q.inv_pn = 0.0; q.inv_pnf = 0.f; q.logP = 0;
    q.bscale = 1.0;
    q.pw = p->opts.pointwise ? 1 : 0;
    q.h1 = 0;
    q.thrs = E * (1.0 - eta / 2.0);
    q.thrsf = (float)q.thrs;
    if (p->ndim == 1) {
      const int64_t P = p1d_len(n);
      q.inv_pn = 1.0 / ((double)P * (double)n);
      q.inv_pnf = (float)q.inv_pn;
      q.logP = ilog2((int)P);
      q.h1 = half_cert_ok(n) ? 1 : 0;
    }
  }
  CK(cudaMemcpyAsync(p->d_prm, p->h_prm, sizeof(ItemParams) * p->batch, cudaMemcpyHostToDevice,
                     p->stream));
}

int read_active(ffcz_plan_s* p) {
  CK(cudaMemcpyAsync(p->h_nactive, p->d_nactive, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return *p->h_nactive;
}

// Commit the pending frequency edits of checks that did not stop the loop.
void edits_finalize(ffcz_plan_s* p) {
  for (auto& dg : p->groups) {
    if (dg.ndim == 1) {   // half spectra of N/2 + 1 <= P/4 + 1 bins per member
      const int64_t slots = (int64_t)dg.P1 * dg.P2 / 4 + 1;
      const unsigned gx = (unsigned)std::min<int64_t>((slots + 255) / 256, 4096);
      k_edits_finalize1<<<dim3(gx, (unsigned)dg.count), 256, 0, p->stream>>>(dg.g, p->d_prm, p->d_st, p->ed_f,
                                                                               p->ed_p, p->ed_t);
      g_launches++;
      continue;
    }
    const int64_t slots = dg.n / 2;
    const unsigned gx = (unsigned)std::min<int64_t>((slots + 255) / 256, 4096);
    k_edits_finalize<<<dim3(gx, (unsigned)dg.count), 256, 0, p->stream>>>(dg.g, p->d_st, p->ed_f, p->ed_p,
                                                                            p->ed_t, slots);
    g_launches++;
  }
}

// Canonical half-spectrum form of the committed frequency edits.
void edits_canon(ffcz_plan_s* p) {
  if (!p->ed_canon) p->ed_canon = (float2*)dalloc(p, sizeof(float2) * std::max<int64_t>(1, p->ed_total[1]));
  if (p->ndim == 1) {   // 1D items record on their half spectra directly
    CK(cudaMemcpyAsync(p->ed_canon, p->ed_f, sizeof(float2) * p->ed_total[1], cudaMemcpyDeviceToDevice, p->stream));
    return;
  }
  for (auto& dg : p->groups) {
    const int64_t nb = (int64_t)dg.Nz * (dg.ndim == 3 ? dg.Ny : 1) * (dg.M + 1);
    const unsigned gx = (unsigned)std::min<int64_t>((nb + 255) / 256, 4096);
    k_edits_canon<<<dim3(gx, (unsigned)dg.count), 256, 0, p->stream>>>(dg.g, p->ed_f, p->ed_canon, dg.d_canon);
    g_launches++;
  }
}

// CompactEdits + QuantizeEdits of both domains of every item into the
// caller's arrays (regions from ed_layout); counts[2 i], counts[2 i + 1] get
// item i's spatial and frequency nonzero counts.
void edits_compact(ffcz_plan_s* p, int m, uint8_t* sf, int32_t* sc, uint8_t* ff, int32_t* fc, int64_t* counts) {
  edits_canon(p);
  const int64_t B = p->batch;
  std::vector<EdRegion<float>> rs(B);
  std::vector<EdRegion<float2>> rf(B);
  int64_t chunks = 0, maxs = 1, maxf = 1;
  for (int64_t i = 0; i < B; ++i) {
    const auto& L = p->ed_layout[i];
    chunks += (L[0] + kEdChunk - 1) / kEdChunk + (L[1] + kEdChunk - 1) / kEdChunk;
    maxs = std::max<int64_t>(maxs, (L[0] + kEdChunk - 1) / kEdChunk);
    maxf = std::max<int64_t>(maxf, (L[1] + kEdChunk - 1) / kEdChunk);
  }
  if (chunks > p->ed_chunk_cap) {
    p->ed_chunks = (int*)dalloc(p, sizeof(int) * chunks);
    p->ed_chunk_cap = chunks;
  }
  if (!p->ed_reg_s) {
    p->ed_reg_s = dalloc(p, sizeof(EdRegion<float>) * B);
    p->ed_reg_f = dalloc(p, sizeof(EdRegion<float2>) * B);
    p->ed_tot = (int64_t*)dalloc(p, sizeof(int64_t) * 2 * B);
  }
  int64_t ch = 0;
  for (int64_t i = 0; i < B; ++i) {
    const auto& L = p->ed_layout[i];
    const float qs = (float)p->h_prm[i].E * ldexpf(1.f, 1 - m);
    const float qf = (float)p->h_prm[i].D * ldexpf(1.f, 1 - m);
    int64_t canon = 0;
    for (int64_t j = 0; j < i; ++j) canon += p->ed_layout[j][1];
    rs[i] = {p->ed_s + p->eoff[i], L[0], sf + L[2], sc + L[3], p->ed_chunks + ch, qs};
    ch += (L[0] + kEdChunk - 1) / kEdChunk;
    rf[i] = {p->ed_canon + canon, L[1], ff + L[4], fc + L[5], p->ed_chunks + ch, qf};
    ch += (L[1] + kEdChunk - 1) / kEdChunk;
  }
  cudaStream_t s = p->stream;
  CK(cudaMemcpyAsync(p->ed_reg_s, rs.data(), sizeof(EdRegion<float>) * B, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p->ed_reg_f, rf.data(), sizeof(EdRegion<float2>) * B, cudaMemcpyHostToDevice, s));
  auto* ds = static_cast<const EdRegion<float>*>(p->ed_reg_s);
  auto* df = static_cast<const EdRegion<float2>*>(p->ed_reg_f);
  k_edits_count<float><<<dim3((unsigned)maxs, (unsigned)B), kEdThreads, 0, s>>>(ds);
  k_edits_scan<float><<<(unsigned)B, 1024, 0, s>>>(ds, p->ed_tot);
  k_edits_scatter<float><<<dim3((unsigned)maxs, (unsigned)B), kEdThreads, 0, s>>>(ds);
  k_edits_count<float2><<<dim3((unsigned)maxf, (unsigned)B), kEdThreads, 0, s>>>(df);
  k_edits_scan<float2><<<(unsigned)B, 1024, 0, s>>>(df, p->ed_tot + B);
  k_edits_scatter<float2><<<dim3((unsigned)maxf, (unsigned)B), kEdThreads, 0, s>>>(df);
  g_launches += 6;
  std::vector<int64_t> tot(2 * B);
  CK(cudaMemcpyAsync(tot.data(), p->ed_tot, sizeof(int64_t) * 2 * B, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if (counts)
    for (int64_t i = 0; i < B; ++i) { counts[2 * i] = tot[i]; counts[2 * i + 1] = tot[B + i]; }
}

// Power-spectrum relative bounds (Sec. V; the mapping is a reading): the
// forward transform of x (x R2C, y FFT, outer-axis FFT as a [Nz][Nmid M]
// view) into the first spectrum buffer, its canonical half spectrum, shell
// sums of |X| and |X|^2, the positive root per shell, one bound per bin.
// The normalisation (x - mean)/mean of the power spectrum cancels out of the
// bound (a relative bound is scale-free and the mean only moves shell 0).
void ps_bounds1(ffcz_plan_s* p, const float* x, const double* rho, float2* out) {
  cudaStream_t s = p->stream;
  int S = 2;
  for (int64_t i = 0; i < p->batch; ++i) S = std::max<int64_t>(S, p->h_prm[i].n / 2 + 2);
  if (!p->ps_acc || p->ps_S < S) {
    p->ps_acc = (double*)dalloc(p, sizeof(double) * 3 * (size_t)S * p->batch);
    p->ps_rho = (double*)dalloc(p, sizeof(double) * p->batch);
    p->ps_S = S;
  }
  S = p->ps_S;
  CK(cudaMemsetAsync(p->ps_acc, 0, sizeof(double) * 3 * (size_t)S * p->batch, s));
  CK(cudaMemcpyAsync(p->ps_rho, rho, sizeof(double) * p->batch, cudaMemcpyHostToDevice, s));
  for (auto& dg : p->groups) {
    // X = DFT(x) by the Bluestein passes, bins k <= N/2 into ed_canon
    Args a = make_args<float>(p, dg, p->B32[0], p->B32[0], p->d_st);
    a.pred = P_ALL;
    a.sel_in = a.sel_out = S_CUR;
    a.pw_e = nullptr; a.pw_f = nullptr;
    a.e = const_cast<float*>(x);
    a.mode = 0;
    col1_args<float>(p, a, dg, OP1_ENTRY);
    launch_col1<float>(dg.P1, dg.w1c, a, dg.P2, dg.count, s);
    row1_args<float>(p, a, dg, OP1_CONV);
    launch_row1<float>(dg.P2, dg.w1r, a, dg.P1, dg.count, s);
    col1_args<float>(p, a, dg, OP1_STOREX);
    a.ed_f = p->ed_canon;
    launch_col1<float>(dg.P1, dg.w1c, a, dg.P2, dg.count, s);
    const unsigned gx = (unsigned)std::min<int64_t>((S + 255) / 256, 1024);
    k_ps_bins1<<<dim3(gx, (unsigned)dg.count), 256, 0, s>>>(dg.g, p->d_prm, p->ed_canon, p->ps_acc, S);
    g_launches++;
  }
  k_ps_roots<<<(unsigned)p->batch, 256, 0, s>>>(p->ps_acc, S, p->ps_rho);
  g_launches++;
  for (auto& dg : p->groups) {
    const unsigned gx = (unsigned)std::min<int64_t>((S + 255) / 256, 1024);
    k_ps_write1<<<dim3(gx, (unsigned)dg.count), 256, 0, s>>>(dg.g, p->d_prm, p->ps_acc, S, out);
    g_launches++;
  }
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
}

void ps_bounds(ffcz_plan_s* p, const float* x, const double* rho, float2* out) {
  cudaStream_t s = p->stream;
  if (!p->ed_canon) p->ed_canon = (float2*)dalloc(p, sizeof(float2) * std::max<int64_t>(1, p->ed_total[1]));
  if (p->ndim == 1) {
    ps_bounds1(p, x, rho, out);
    return;
  }
  int S = 1;
  for (auto& dg : p->groups) {
    const double r = std::sqrt((double)dg.M * dg.M + std::pow(dg.Nz / 2, 2.0) +
                               (dg.ndim == 3 ? std::pow(dg.Ny / 2, 2.0) : 0.0));
    S = std::max(S, (int)std::ceil(r) + 2);
  }
  if (!p->ps_acc) {
    p->ps_acc = (double*)dalloc(p, sizeof(double) * 3 * (size_t)S * p->batch);
    p->ps_rho = (double*)dalloc(p, sizeof(double) * p->batch);
    p->ps_S = S;
  }
  double* acc = p->ps_acc;
  double* d_rho = p->ps_rho;
  CK(cudaMemsetAsync(acc, 0, sizeof(double) * 3 * (size_t)S * p->batch, s));
  CK(cudaMemcpyAsync(d_rho, rho, sizeof(double) * p->batch, cudaMemcpyHostToDevice, s));
  for (auto& dg : p->groups) {
    const int Nmid = dg.ndim == 3 ? dg.Ny : 1;
    Args a = make_args<float>(p, dg, p->B32[0], p->B32[0], p->d_st);
    a.pred = P_ALL;
    a.sel_in = a.sel_out = S_CUR;
    a.pw_e = nullptr; a.pw_f = nullptr;
    tabs_x<float>(p, a, dg);
    a.e = const_cast<float*>(x);
    a.mode = 0;
    launch_x<float>(XFWD, dg.M, dg.wx, a, dg.rows, dg.count, s);
    if (dg.ndim == 3) {
      set_tw<float>(a, p->tb, dg.Ny);
      launch_axis<float, -1>(dg.Ny, dg.wa, a, dg.Nz, dg.M, dg.count, s);
    }
    Args az = a;
    az.g.Nz = 1;
    az.g.M = Nmid * dg.M;
    set_tw<float>(az, p->tb, dg.Nz);
    launch_axis<float, -1>(dg.Nz, dg.wa, az, 1, Nmid * dg.M, dg.count, s);
    const int64_t nb = (int64_t)dg.Nz * Nmid * (dg.M + 1);
    const unsigned gx = (unsigned)std::min<int64_t>((nb + 255) / 256, 1024);
    k_edits_canon<<<dim3(gx, (unsigned)dg.count), 256, 0, s>>>(dg.g, static_cast<const float2*>(p->B32[0]),
                                                                p->ed_canon, dg.d_canon);
    const size_t hs = sizeof(double) * 3 * S;
    if (hs > 48 * 1024) CK(cudaFuncSetAttribute(k_ps_shells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs));
    k_ps_shells<<<dim3(std::min<unsigned>(gx, 296), (unsigned)dg.count), 256, hs, s>>>(dg.g, p->ed_canon, acc, S);
    g_launches += 2;
  }
  k_ps_roots<<<(unsigned)p->batch, 256, 0, s>>>(acc, S, d_rho);
  g_launches++;
  for (auto& dg : p->groups) {
    const int64_t nb = (int64_t)dg.Nz * (dg.ndim == 3 ? dg.Ny : 1) * (dg.M + 1);
    const unsigned gx = (unsigned)std::min<int64_t>((nb + 255) / 256, 1024);
    k_ps_write<<<dim3(gx, (unsigned)dg.count), 256, 0, s>>>(dg.g, acc, S, out);
    g_launches++;
  }
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
}

// Applying edits (Sec. IV-B): x_hat += S~ + IFFT(F~) from the stored form
// (flags and codes at the offsets of ed_layout).  Spatial codes are added in
// place; frequency codes are expanded to the canonical half spectrum, packed,
// and transformed back by the inverse passes (outer axis, middle axis, x C2R
// with 1/N), the last of which adds its result to x_hat.
void apply_edits(ffcz_plan_s* p, float* xhat, int m, const uint8_t* sf, const int32_t* sc,
                 const uint8_t* ff, const int32_t* fc) {
  const int64_t B = p->batch;
  if (!p->ed_canon) p->ed_canon = (float2*)dalloc(p, sizeof(float2) * std::max<int64_t>(1, p->ed_total[1]));
  int64_t chunks = 0, maxs = 1, maxf = 1;
  for (int64_t i = 0; i < B; ++i) {
    const auto& L = p->ed_layout[i];
    chunks += (L[0] + kEdChunk - 1) / kEdChunk + (L[1] + kEdChunk - 1) / kEdChunk;
    maxs = std::max<int64_t>(maxs, (L[0] + kEdChunk - 1) / kEdChunk);
    maxf = std::max<int64_t>(maxf, (L[1] + kEdChunk - 1) / kEdChunk);
  }
  if (chunks > p->ed_chunk_cap) {
    p->ed_chunks = (int*)dalloc(p, sizeof(int) * chunks);
    p->ed_chunk_cap = chunks;
  }
  if (!p->ap_reg) p->ap_reg = dalloc(p, sizeof(ApRegion) * 2 * B);
  std::vector<ApRegion> r(2 * B);
  int64_t ch = 0, canon = 0;
  for (int64_t i = 0; i < B; ++i) {
    const auto& L = p->ed_layout[i];
    const float qs = (float)p->h_prm[i].E * ldexpf(1.f, 1 - m);
    const float qf = (float)p->h_prm[i].D * ldexpf(1.f, 1 - m);
    r[i] = {sf + L[2], sc + L[3], L[0], p->ed_chunks + ch, qs, xhat + p->eoff[i], nullptr};
    ch += (L[0] + kEdChunk - 1) / kEdChunk;
    r[B + i] = {ff + L[4], fc + L[5], L[1], p->ed_chunks + ch, qf, nullptr, p->ed_canon + canon};
    ch += (L[1] + kEdChunk - 1) / kEdChunk;
    canon += L[1];
  }
  cudaStream_t s = p->stream;
  CK(cudaMemcpyAsync(p->ap_reg, r.data(), sizeof(ApRegion) * 2 * B, cudaMemcpyHostToDevice, s));
  auto* rs = static_cast<const ApRegion*>(p->ap_reg);
  auto* rf = rs + B;
  k_apply_count<<<dim3((unsigned)maxs, (unsigned)B), kEdThreads, 0, s>>>(rs);
  k_apply_scan<<<(unsigned)B, 1024, 0, s>>>(rs);
  k_apply_expand<false><<<dim3((unsigned)maxs, (unsigned)B), kEdThreads, 0, s>>>(rs);
  k_apply_count<<<dim3((unsigned)maxf, (unsigned)B), kEdThreads, 0, s>>>(rf);
  k_apply_scan<<<(unsigned)B, 1024, 0, s>>>(rf);
  k_apply_expand<true><<<dim3((unsigned)maxf, (unsigned)B), kEdThreads, 0, s>>>(rf);
  g_launches += 6;
  if (p->ndim == 1) {
    // x_hat += IDFT(F): the half spectrum times the chirp, forward column
    // step; row pass with conj Bt; inverse column step, x = Re(b c) / (P N)
    // added to x_hat
    for (auto& dg : p->groups) {
      Args a = make_args<float>(p, dg, p->B32[0], p->B32[0], p->d_st);
      a.pred = P_ALL;
      a.sel_in = a.sel_out = S_CUR;
      a.pw_e = nullptr; a.pw_f = nullptr;
      a.ed_f = p->ed_canon;
      col1_args<float>(p, a, dg, OP1_LOADX);
      a.mode = 0;
      launch_col1<float>(dg.P1, dg.w1c, a, dg.P2, dg.count, s);
      a.ed_f = nullptr;
      row1_args<float>(p, a, dg, OP1_CONVC);
      launch_row1<float>(dg.P2, dg.w1r, a, dg.P1, dg.count, s);
      col1_args<float>(p, a, dg, OP1_EXIT);
      a.e = xhat;
      a.mode = M_ACC;
      launch_col1<float>(dg.P1, dg.w1c, a, dg.P2, dg.count, s);
    }
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    return;
  }
  for (auto& dg : p->groups) {
    const int Nmid = dg.ndim == 3 ? dg.Ny : 1;
    const int64_t slots = (int64_t)dg.Nz * Nmid * dg.M;
    const unsigned gx = (unsigned)std::min<int64_t>((slots + 255) / 256, 4096);
    k_edits_pack<<<dim3(gx, (unsigned)dg.count), 256, 0, s>>>(dg.g, p->ed_canon, dg.d_canon,
                                                              static_cast<float2*>(p->B32[0]));
    g_launches++;
    Args a = make_args<float>(p, dg, p->B32[0], p->B32[0], p->d_st);
    a.pred = P_ALL;
    a.sel_in = a.sel_out = S_CUR;
    // outer axis as a [Nz][Nmid M] view (pencils of length Nz, stride Nmid M)
    Args az = a;
    az.g.Nz = 1;
    az.g.M = Nmid * dg.M;
    set_tw<float>(az, p->tb, dg.Nz);
    launch_axis<float, +1>(dg.Nz, dg.wa, az, 1, Nmid * dg.M, dg.count, s);
    if (dg.ndim == 3) {
      set_tw<float>(a, p->tb, dg.Ny);
      launch_axis<float, +1>(dg.Ny, dg.wa, a, dg.Nz, dg.M, dg.count, s);
    }
    tabs_x<float>(p, a, dg);
    a.e = xhat;
    a.mode = M_ACC;
    launch_x<float>(XEXIT, dg.M, dg.wx, a, dg.rows, dg.count, s);
  }
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
}

// 16-bit storage of the codes of 2 B regions: narrowing (int32 -> int16 and
// the escaped values) or widening (back to int32; every region must hold
// exactly its nwide escapes).  esc[r] receives region r's escape count.
void codes_convert(ffcz_plan_s* p, std::vector<CodeRegion>& rg, bool narrow, std::vector<int64_t>& esc) {
  const int64_t R = (int64_t)rg.size();
  int64_t chunks = 0, maxc = 1;
  for (auto& r : rg) {
    const int64_t c = (r.n + kEdChunk - 1) / kEdChunk;
    chunks += c;
    maxc = std::max(maxc, c);
  }
  if (chunks > p->cd_chunk_cap) {
    p->cd_chunks = (int*)dalloc(p, sizeof(int) * std::max<int64_t>(1, chunks));
    p->cd_chunk_cap = chunks;
  }
  if (!p->cd_reg) {
    p->cd_reg = dalloc(p, sizeof(CodeRegion) * R);
    p->cd_tot = (int64_t*)dalloc(p, sizeof(int64_t) * R);
  }
  int64_t ch = 0;
  for (auto& r : rg) {
    r.chunks = p->cd_chunks + ch;
    ch += (r.n + kEdChunk - 1) / kEdChunk;
  }
  cudaStream_t s = p->stream;
  CK(cudaMemcpyAsync(p->cd_reg, rg.data(), sizeof(CodeRegion) * R, cudaMemcpyHostToDevice, s));
  auto* d = static_cast<const CodeRegion*>(p->cd_reg);
  if (narrow) k_codes_count<true><<<dim3((unsigned)maxc, (unsigned)R), kEdThreads, 0, s>>>(d);
  else k_codes_count<false><<<dim3((unsigned)maxc, (unsigned)R), kEdThreads, 0, s>>>(d);
  k_codes_scan<<<(unsigned)R, 1024, 0, s>>>(d, p->cd_tot);
  g_launches += 2;
  esc.assign(R, 0);
  CK(cudaMemcpyAsync(esc.data(), p->cd_tot, sizeof(int64_t) * R, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (!narrow)
    for (int64_t r = 0; r < R; ++r)
      if (esc[r] != rg[r].nwide) fail(FFCZ_ERR_INVALID, "escape count of the 16-bit codes differs from counts");
  if (narrow) k_codes_scatter<true><<<dim3((unsigned)maxc, (unsigned)R), kEdThreads, 0, s>>>(d);
  else k_codes_scatter<false><<<dim3((unsigned)maxc, (unsigned)R), kEdThreads, 0, s>>>(d);
  g_launches++;
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
}

int32_t* codes32(ffcz_plan_s* p) {
  if (!p->cd_c32)
    p->cd_c32 = (int32_t*)dalloc(p, sizeof(int32_t) * std::max<int64_t>(1, p->ed_total[3] + p->ed_total[5]));
  return p->cd_c32;
}

// CompactEdits + QuantizeEdits with the codes stored in 16 bits; counts (4
// per item): nonzero spatial components, nonzero bins, spatial escapes,
// frequency escapes.
void edits_compact16(ffcz_plan_s* p, int m, uint8_t* sf, int16_t* sc, int32_t* sw, uint8_t* ff, int16_t* fc,
                     int32_t* fw, int64_t* counts) {
  const int64_t B = p->batch;
  int32_t* s32 = codes32(p);
  int32_t* f32 = s32 + p->ed_total[3];
  std::vector<int64_t> nz(2 * B), esc;
  edits_compact(p, m, sf, s32, ff, f32, nz.data());
  std::vector<CodeRegion> rg(2 * B);
  for (int64_t i = 0; i < B; ++i) {
    const auto& L = p->ed_layout[i];
    rg[i] = {s32 + L[3], sc + L[3], sw + L[3], nz[2 * i], 0, nullptr};
    rg[B + i] = {f32 + L[5], fc + L[5], fw + L[5], 2 * nz[2 * i + 1], 0, nullptr};
  }
  codes_convert(p, rg, true, esc);
  if (counts)
    for (int64_t i = 0; i < B; ++i) {
      counts[4 * i] = nz[2 * i];
      counts[4 * i + 1] = nz[2 * i + 1];
      counts[4 * i + 2] = esc[i];
      counts[4 * i + 3] = esc[B + i];
    }
}

// The decompression side from the 16-bit form: the codes widened to int32,
// then applied as from ffcz_edits_compact's form.
void apply_edits16(ffcz_plan_s* p, float* xhat, int m, const uint8_t* sf, const int16_t* sc, const int32_t* sw,
                   const uint8_t* ff, const int16_t* fc, const int32_t* fw, const int64_t* counts) {
  const int64_t B = p->batch;
  for (int64_t i = 0; i < B; ++i) {
    const auto& L = p->ed_layout[i];
    const int64_t ns = counts[4 * i], nf = counts[4 * i + 1], es = counts[4 * i + 2], ef = counts[4 * i + 3];
    if (ns < 0 || ns > L[0] || nf < 0 || nf > L[1] || es < 0 || es > ns || ef < 0 || ef > 2 * nf)
      fail(FFCZ_ERR_INVALID, "edit counts out of range");
  }
  int32_t* s32 = codes32(p);
  int32_t* f32 = s32 + p->ed_total[3];
  std::vector<CodeRegion> rg(2 * B);
  for (int64_t i = 0; i < B; ++i) {
    const auto& L = p->ed_layout[i];
    rg[i] = {s32 + L[3], const_cast<int16_t*>(sc) + L[3], const_cast<int32_t*>(sw) + L[3], counts[4 * i],
             counts[4 * i + 2], nullptr};
    rg[B + i] = {f32 + L[5], const_cast<int16_t*>(fc) + L[5], const_cast<int32_t*>(fw) + L[5],
                 2 * counts[4 * i + 1], counts[4 * i + 3], nullptr};
  }
  std::vector<int64_t> esc;
  codes_convert(p, rg, false, esc);
  apply_edits(p, xhat, m, sf, s32, ff, f32);
}

template <typename T>
void run_loop(ffcz_plan_s* p, float* e, bool only_uncert) {
  p->ed_on = p->opts.edits != 0;   // the loop's kernels record edits
  // the projection variant runs in the float32 loop; FP64 repairs use Alg. 1
  p->pv_on = sizeof(T) == 4 && p->opts.method != PV_POCS;
  struct Off { ffcz_plan_s* p; ~Off() { p->ed_on = false; p->pv_on = false; } } off_{p};
  LoopBufs B = loop_bufs<T>(p);
  CK(cudaMemsetAsync(p->d_nactive, 0, sizeof(int), p->stream));
  k_init<<<(unsigned)((p->batch + 255) / 256), 256, 0, p->stream>>>(p->d_st, (int)p->batch,
                                                                   only_uncert ? 1 : 0, p->d_nactive);
  g_launches++;
  entry<T>(p, B, e, !only_uncert, p->stream);
  if (sizeof(T) == 4 && p->ck_rec)   // checkpoint t = 0: e0 after the pre-clip
    CK(cudaMemcpyAsync(p->bw_ck, e, sizeof(float) * p->total, cudaMemcpyDeviceToDevice, p->stream));
  const int cap = p->h_prm[0].max_iters;   // no item iterates past it
  if (p->opts.use_graph == 2 && !p->prof && cap > 0) {
    // the whole loop on the device (conditional WHILE node); graphs are
    // rebuilt when the cap changes
    const int slot = sizeof(T) == 4 ? 0 : 1;
    const int ckk = ((sizeof(T) == 4 && p->ck_rec) ? 1 : 0) + (keep_masks_rec<T>(p) ? 2 : 0);
    const auto key = std::make_pair(-(int)sizeof(T), ckk);
    if (p->while_cap[slot][ckk] != cap && p->graphs.count(key)) {
      cudaGraphExecDestroy(p->graphs[key]);
      p->graphs.erase(key);
    }
    run_while_graph<T>(p, B, cap);
    // the executed-body count is read with the stats at the end of the call
    // (launch accounting only)
    CK(cudaMemcpyAsync(p->h_loopcount, p->d_loopcount, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    p->count_pending = true;
  } else {
    int chunk = 1, launched = 0;
    const int cmax = std::max(1, p->opts.chunk);
    while (launched < cap && read_active(p) > 0) {
      const int c = std::min(chunk, cap - launched);
      run_chunk<T>(p, B, c);
      launched += c;
      chunk = std::min(chunk * 2, cmax);
    }
  }
  exit_pass<T>(p, B, e, p->stream);
  if (p->ed_on) edits_finalize(p);
}

// Tables of the N/2-point certification (1D, even N): chirps of length
// N/2, Bt = FFT_{P/2} of their wrapped chirp, the twiddles W_N^k and the
// buffer of Z (float64).
void build_half(ffcz_plan_s* p) {
  if (p->Bz || p->hgroups.empty()) return;
  cudaStream_t s = p->stream;
  p->ch64h = dalloc(p, sizeof(double2) * p->total);
  p->Bt64h = dalloc(p, sizeof(double2) * p->total_c);
  p->Bz = dalloc(p, sizeof(double2) * p->total_c);
  p->rtw = (double2*)dalloc(p, sizeof(double2) * std::max<int64_t>(1, p->ed_total[1]));
  for (auto& hg : p->hgroups) {
    k1_chirp_table<double><<<dim3(64, (unsigned)hg.count), 256, 0, s>>>(hg.g, p->d_prm,
                                                                      static_cast<double2*>(p->ch64h), 1);
    k1_rtw<<<dim3(64, (unsigned)hg.count), 256, 0, s>>>(hg.g, p->d_prm, p->rtw);
    g_launches += 2;
    Args a = make_args<double>(p, hg, p->Bt64h, p->Bt64h, p->d_st);
    a.pred = P_ALL;
    a.half1 = 1;
    col1_args<double>(p, a, hg, OP1_FILTER);
    a.chirp = p->ch64h;
    launch_col1<double>(hg.P1, hg.w1c, a, hg.P2, hg.count, s);
    row1_args<double>(p, a, hg, OP1_FWD);
    launch_row1<double>(hg.P2, hg.w1r, a, hg.P1, hg.count, s);
  }
}

// st: the state the certification reads and writes (default the loop's);
// x_done / y_done: the x pass (and the y pass) already ran into the FP64
// buffer (host entry point).
void certify(ffcz_plan_s* p, const float* e, bool repair_round, ItemState* st = nullptr, bool x_done = false,
             bool y_done = false) {
  ItemState* S = st ? st : p->d_st;
  if (!p->Bc) p->Bc = dalloc(p, (size_t)p->total_c * sizeof(double2));
  if (p->ndim == 1 && !p->Bt64) build_bt<double>(p);
  if (p->ndim == 1) {
    // odd (and short) lengths: the N-point transform; even lengths: the
    // N/2-point transform of x_2n + i x_2n+1 and the real-input post-processing
    const bool halves = !p->hgroups.empty();
    if (halves) build_half(p);
    const int pred = repair_round ? P_UNCERT : P_ALL;
    for (auto& dg : p->groups) {
      Args a = make_args<double>(p, dg, p->Bc, p->Bc, S);
      a.pred = pred;
      a.half1 = halves ? 2 : 0;
      a.e = const_cast<float*>(e);
      col1_args<double>(p, a, dg, OP1_ENTRY);
      a.mode = M_MEASURE;
      launch_col1<double>(dg.P1, dg.w1c, a, dg.P2, dg.count, p->stream);
      row1_args<double>(p, a, dg, OP1_CONV);
      a.mode = 0;
      launch_row1<double>(dg.P2, dg.w1r, a, dg.P1, dg.count, p->stream);
      col1_args<double>(p, a, dg, OP1_FCLIP);
      a.mode = M_NOWRITE;
      launch_col1<double>(dg.P1, dg.w1c, a, dg.P2, dg.count, p->stream);
    }
    for (auto& hg : p->hgroups) {
      Args a = make_args<double>(p, hg, p->Bc, p->Bc, S);
      a.pred = pred;
      a.half1 = 1;
      a.e = const_cast<float*>(e);
      col1_args<double>(p, a, hg, OP1_ENTRY);
      a.chirp = p->ch64h;
      a.mode = M_MEASURE;
      launch_col1<double>(hg.P1, hg.w1c, a, hg.P2, hg.count, p->stream);
      row1_args<double>(p, a, hg, OP1_CONV);
      a.bt = p->Bt64h;
      a.mode = 0;
      launch_row1<double>(hg.P2, hg.w1r, a, hg.P1, hg.count, p->stream);
      col1_args<double>(p, a, hg, OP1_ZOUT);
      a.chirp = p->ch64h;
      a.zout = p->Bz;
      launch_col1<double>(hg.P1, hg.w1c, a, hg.P2, hg.count, p->stream);
      const unsigned gx = (unsigned)std::min<int64_t>(((int64_t)hg.P1 * hg.P2 / 2 + 256) / 256, 1024);
      k1_rpost<<<dim3(gx, (unsigned)hg.count), 256, 0, p->stream>>>(
          hg.g, p->d_prm, S, pred, static_cast<const double2*>(p->Bz), p->rtw,
          p->opts.pointwise ? p->pw_f : nullptr);
      g_launches++;
    }
  }
  for (auto& dg : p->groups) {
    if (p->ndim == 1) break;
    Args a = make_args<double>(p, dg, p->Bc, p->Bc, S);
    a.pred = repair_round ? P_UNCERT : P_ALL;
    tabs_x<double>(p, a, dg);
    a.e = const_cast<float*>(e);
    a.mode = M_MEASURE;
    if (!x_done) launch_x<double>(XCERT, dg.M, dg.wx, a, dg.rows, dg.count, p->stream);
    if (dg.ndim == 3 && !y_done) {
      set_tw<double>(a, p->tb, dg.Ny);
      a.mode = 0;
      launch_axis<double, -1>(dg.Ny, dg.wa, a, dg.Nz, dg.M, dg.count, p->stream);
    }
    set_tw<double>(a, p->tb, dg.Nz);
    a.mode = M_NOWRITE;
    launch_chk<double>(dg.Nz, dg.wc, a, dg.ndim == 3 ? dg.Ny : 1, dg.M, dg.count, p->stream);
  }
  // 2D/3D certification transforms return 2 delta (XCERT)
  k_certify<<<(unsigned)((p->batch + 255) / 256), 256, 0, p->stream>>>(
      p->d_prm, S, (int)p->batch, repair_round ? 1 : 0, p->ndim == 1 ? 1.0 : 0.5);
  g_launches++;
}

// Certification results computed in a side state (the host entry point's
// x pass during the upload) adopted by the loop's state.
__global__ void k_cert_adopt(ItemState* st, const ItemState* sc, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  st[i].certified = sc[i].certified;
  st[i].v64 = sc[i].v64;
  st[i].emax64 = sc[i].emax64;
  st[i].bound64 = sc[i].bound64;
}

// Reset the certification accumulators (they are shared with the loop).
__global__ void k_cert_reset(ItemState* st, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  st[i].vbits = 0ull;
  st[i].emaxbits = 0ull;
  st[i].sumsq = 0.0;
}

void cert_reset(ffcz_plan_s* p) {
  k_cert_reset<<<(unsigned)((p->batch + 255) / 256), 256, 0, p->stream>>>(p->d_st, (int)p->batch);
  g_launches++;
}

__global__ void k_set_repairs(ItemState* st, int n, int round) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!st[i].certified) st[i].repairs = round;
}

void check_dev_err(ffcz_plan_s* p) {
  if (*p->h_err == DERR_NONE) return;
  const int e = *p->h_err;
  *p->h_err = 0;
  CK(cudaMemsetAsync(p->d_err, 0, sizeof(int), p->stream));
  if (e == DERR_TMA_TIMEOUT) fail(FFCZ_ERR_TIMEOUT, "a TMA tile load did not complete within its poll limit");
  fail(FFCZ_ERR_CUDA, "a TMA staging buffer was not 128-byte aligned");
}

void fill_stats(ffcz_plan_s* p, ffcz_stats* out, float ms, float ms_cert, bool certified_run) {
  CK(cudaMemcpyAsync(p->h_st, p->d_st, sizeof(ItemState) * p->batch, cudaMemcpyDeviceToHost,
                     p->stream));
  CK(cudaMemcpyAsync(p->h_err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  check_dev_err(p);
  if (p->count_pending) {
    g_launches += (int64_t)(*p->h_loopcount) * p->pending_bodies_per;
    p->count_pending = false;
  }
  if (!out) return;
  for (int64_t i = 0; i < p->batch; ++i) {
    const ItemState& s = p->h_st[i];
    const ItemParams& q = p->h_prm[i];
    ffcz_stats& o = out[i];
    memset(&o, 0, sizeof(o));
    o.status = s.status;
    o.iters = s.t;
    o.repairs = s.repairs;
    o.certified = certified_run ? s.certified : 0;
    o.preclipped = s.preclip;
    o.f_ratio = s.f_ratio;
    if (certified_run) {
      o.s_ratio = s.emax64 / q.E;
      o.f_margin64 = 1.0 - (s.v64 + s.bound64) / q.D;
      o.s_margin64 = 1.0 - s.emax64 / q.E;
    }
    o.active_s = (int64_t)s.last_act_s;
    o.active_f = (int64_t)s.last_act_f;
    o.ms_total = ms;
    o.ms_cert = ms_cert;
  }
}

ffcz_status worst_status(ffcz_plan_s* p, bool certified_run) {
  int worst = 0;
  auto rank = [](int s) { return s == 0 ? 0 : s == 4 ? 1 : s == 5 ? 2 : s == 6 ? 3 : 4; };
  for (int64_t i = 0; i < p->batch; ++i) {
    int s = p->h_st[i].status;
    if (s == 0 && certified_run && !p->h_st[i].certified) s = FFCZ_ERR_CERT_FAILED;
    if (rank(s) > rank(worst)) worst = s;
  }
  return (ffcz_status)worst;
}

template <typename F>
ffcz_status guarded(F&& f) {
  try {
    g_err.clear();
    return f();
  } catch (const Fail& x) {
    return x.s;
  } catch (const std::exception& x) {
    g_err = x.what();
    return FFCZ_ERR_CUDA;
  } catch (...) {
    g_err = "unknown error";
    return FFCZ_ERR_CUDA;
  }
}

void free_plan(ffcz_plan_s* p) {
  for (auto& kv : p->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& x : p->pend) { cudaEventDestroy(x.a); cudaEventDestroy(x.b); }
  for (auto e : p->evpool) cudaEventDestroy(e);
  for (void* a : p->allocs) cudaFree(a);
  if (p->h_nactive) cudaFreeHost(p->h_nactive);
  if (p->h_loopcount) cudaFreeHost(p->h_loopcount);
  if (p->h_err) cudaFreeHost(p->h_err);
  if (p->h_st) cudaFreeHost(p->h_st);
  if (p->h_prm) cudaFreeHost(p->h_prm);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  if (p->ev2) cudaEventDestroy(p->ev2);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
  if (p->ev_copy) cudaEventDestroy(p->ev_copy);
  if (p->spec_stream) cudaStreamDestroy(p->spec_stream);
  for (auto ev : p->ev_chunks) cudaEventDestroy(ev);
  if (p->ev_spec) cudaEventDestroy(p->ev_spec);
  delete p;
}

struct ProfOn {
  ffcz_plan_s* p;
  explicit ProfOn(ffcz_plan_s* p_) : p(p_) {
    g_prof = p->prof ? p : nullptr;
  }
  ~ProfOn() {
    if (g_prof) {
      try { cudaStreamSynchronize(p->stream); prof_collect(p); } catch (...) {}
    }
    g_prof = nullptr;
  }
};

// Validate the plan's copies of the pointwise bounds and set, per item,
// bscale = 1 / min_k Delta_k (the certification's bound is absolute while the
// violations are ratios).
void pw_prepare(ffcz_plan_s* p) {
  cudaStream_t s = p->stream;
  CK(cudaMemsetAsync(p->pw_bad, 0, sizeof(int), s));
  std::vector<unsigned int> inf(p->batch, 0x7f800000u);
  CK(cudaMemcpyAsync(p->pw_min, inf.data(), sizeof(unsigned int) * p->batch, cudaMemcpyHostToDevice, s));
  for (auto& dg : p->groups) {
    if (dg.ndim == 1) {   // members of uneven length: N and N/2 + 1 bins read per member
      k_pw_check1<<<dim3(64, (unsigned)dg.count), 256, 0, s>>>(dg.g, p->d_prm, p->pw_e, p->pw_f, p->pw_min,
                                                               p->pw_bad);
      g_launches++;
      continue;
    }
    const int64_t nb = (int64_t)dg.Nz * (dg.ndim == 3 ? dg.Ny : 1) * (dg.M + 1);
    const unsigned gx = (unsigned)std::min<int64_t>((std::max(dg.n, nb) + 255) / 256, 2048);
    k_pw_check<<<dim3(gx, (unsigned)dg.count), 256, 0, s>>>(dg.g, p->pw_e, p->pw_f, dg.n, nb, p->pw_min,
                                                            p->pw_bad);
    g_launches++;
    const unsigned gp = (unsigned)std::min<int64_t>((nb + 255) / 256, 2048);
    k_pw_pack<<<dim3(gp, (unsigned)dg.count), 256, 0, s>>>(dg.g, p->pw_f, p->pw_fp,
                                                           reinterpret_cast<float2*>(p->pw_f0), nb);
    g_launches++;
  }
  k_pw_scale<<<(unsigned)((p->batch + 255) / 256), 256, 0, s>>>(p->d_prm, p->pw_min, (int)p->batch);
  g_launches++;
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, p->pw_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad) fail(FFCZ_ERR_INVALID, "pointwise bounds must be finite and > 0");
}

// host_out (host-buffer entry point): the corrected field is copied back on a
// second stream as soon as the loop is done, overlapping the certification,
// which only reads e; a repair round waits for that copy and the field is
// copied again at the end.
// Host-buffer entry point: upload the field in chunks of whole CTA rows on
// the copy stream and run the FP64 certification's x pass on each chunk as
// it lands (on a third stream, into the FP64 buffer and the side state
// d_stc), so the transfer hides most of that pass; for 3D items the chunks
// are whole z-planes and the certification's y pass runs on each as well.
// The loop's stream waits for the last chunk only.  Single-item 2D/3D plans
// with certification.
bool spec_upload(ffcz_plan_s* p, float* e_dev, const float* host) {
  if (p->batch != 1 || p->ndim < 2 || !p->opts.certify || p->opts.pointwise) return false;
  const DevGroup& dg = p->groups[0];
  if (!p->copy_stream) {
    CK(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&p->ev_copy, cudaEventDisableTiming));
  }
  constexpr int K = 8;
  if (!p->spec_stream) {
    CK(cudaStreamCreateWithFlags(&p->spec_stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&p->ev_spec, cudaEventDisableTiming));
    p->ev_chunks.resize(K + 1);
    for (auto& ev : p->ev_chunks) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  if (!p->d_stc) p->d_stc = (ItemState*)dalloc(p, sizeof(ItemState) * p->batch);
  if (!p->Bc) p->Bc = dalloc(p, (size_t)p->total_c * sizeof(double2));
  // everything earlier on the plan's stream (a previous call) is done with
  // the staging and FP64 buffers before the chunks start
  CK(cudaEventRecord(p->ev_chunks[K], p->stream));
  CK(cudaStreamWaitEvent(p->copy_stream, p->ev_chunks[K], 0));
  CK(cudaStreamWaitEvent(p->spec_stream, p->ev_chunks[K], 0));
  CK(cudaMemsetAsync(p->d_stc, 0, sizeof(ItemState) * p->batch, p->spec_stream));
  // rows of one CTA of the FP64 x pass (tiles of row_w1(M) rows, G per CTA)
  const int W = row_w1(dg.M), tpt = f2_nt(dg.M) * W, rpc = (tpt >= 128 ? 1 : 128 / tpt) * W;
  const int64_t rows = dg.rows, Nx = 2 * (int64_t)dg.M;
  const int64_t unit = dg.ndim == 3 ? std::lcm((int64_t)rpc, (int64_t)dg.Ny) : rpc;
  const int64_t crow = ((rows + K - 1) / K + unit - 1) / unit * unit;
  const int tpr_y = dg.M / kAxisW64;   // y-pass tiles per z-plane
  int c = 0;
  for (int64_t r0 = 0; r0 < rows; r0 += crow, ++c) {
    const int64_t nr = std::min(crow, rows - r0);
    CK(cudaMemcpyAsync(e_dev + r0 * Nx, host + r0 * Nx, sizeof(float) * nr * Nx, cudaMemcpyHostToDevice,
                       p->copy_stream));
    CK(cudaEventRecord(p->ev_chunks[c], p->copy_stream));
    CK(cudaStreamWaitEvent(p->spec_stream, p->ev_chunks[c], 0));
    Args a = make_args<double>(p, dg, p->Bc, p->Bc, p->d_stc);
    a.pred = P_ALL;
    tabs_x<double>(p, a, dg);
    a.e = e_dev;
    a.mode = M_MEASURE;
    a.tile0 = (int)(r0 / W);
    launch_x<double>(XCERT, dg.M, dg.wx, a, nr, 1, p->spec_stream);
    if (dg.ndim == 3) {   // planes z0 .. z1 - 1
      const int z0 = (int)(r0 / dg.Ny), z1 = (int)((r0 + nr) / dg.Ny);
      set_tw<double>(a, p->tb, dg.Ny);
      a.mode = 0;
      a.tile0 = z0 * tpr_y;
      a.tile1 = z1 * tpr_y;
      launch_axis<double, -1>(dg.Ny, dg.wa, a, z1 - z0, dg.M, 1, p->spec_stream);
    }
  }
  p->spec_y = dg.ndim == 3;
  CK(cudaEventRecord(p->ev_spec, p->spec_stream));
  CK(cudaStreamWaitEvent(p->stream, p->ev_chunks[c - 1], 0));   // the loop needs the whole field
  return true;
}

// After the loop: if it stopped at 0 iterations without a pre-clip, the
// field is the uploaded one and the certification continues from the x pass
// of spec_upload (y and z passes, the check, adopted by the loop's state).
bool spec_adopt(ffcz_plan_s* p, const float* e) {
  CK(cudaStreamWaitEvent(p->stream, p->ev_spec, 0));
  CK(cudaMemcpyAsync(p->h_st, p->d_st, sizeof(ItemState) * p->batch, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  for (int64_t i = 0; i < p->batch; ++i)
    if (p->h_st[i].t != 0 || p->h_st[i].preclip || p->h_st[i].status != 0) return false;
  certify(p, e, false, p->d_stc, true, p->spec_y);
  k_cert_adopt<<<(unsigned)((p->batch + 255) / 256), 256, 0, p->stream>>>(p->d_st, p->d_stc, (int)p->batch);
  g_launches++;
  return true;
}

ffcz_status correct_impl(ffcz_plan_s* p, float* e, const double* eps_s, const double* eps_f,
                         ffcz_stats* stats, float* host_out = nullptr, bool spec_x = false) {
  if (!e || !eps_s || !eps_f) fail(FFCZ_ERR_INVALID, "null pointer argument");
  ProfOn prof_on(p);
  CK(cudaSetDevice(p->device));
  upload_params(p, eps_s, eps_f, p->opts.min_iters, p->opts.max_iters);
  if (p->opts.pointwise) pw_prepare(p);
  CK(cudaEventRecord(p->ev0, p->stream));
  if (p->opts.edits) {
    CK(cudaMemsetAsync(p->ed_s, 0, sizeof(float) * p->total, p->stream));
    CK(cudaMemsetAsync(p->ed_f, 0, sizeof(float2) * p->total_c, p->stream));
    CK(cudaMemsetAsync(p->ed_p, 0, sizeof(float2) * p->total_c, p->stream));
    CK(cudaMemsetAsync(p->ed_t, 0, sizeof(int) * p->total_c, p->stream));
  }
  if (p->opts.precision == 64) run_loop<double>(p, e, false);
  else run_loop<float>(p, e, false);
  CK(cudaEventRecord(p->ev1, p->stream));
  bool cert = p->opts.certify != 0;
  // adopted: the loop left the uploaded field unchanged (0 iterations, no
  // pre-clip), so the host buffer already holds the result
  const bool adopted = cert && spec_x && spec_adopt(p, e);
  if (cert && !adopted) {
    cert_reset(p);
    certify(p, e, false);
  }
  bool recopy = false;
  int copies = 0;
  if (host_out && !adopted) {
    copies = 1;
    if (!p->copy_stream) {
      CK(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&p->ev_copy, cudaEventDisableTiming));
    }
    CK(cudaStreamWaitEvent(p->copy_stream, p->ev1, 0));
    CK(cudaMemcpyAsync(host_out, e, sizeof(float) * p->total, cudaMemcpyDeviceToHost, p->copy_stream));
    CK(cudaEventRecord(p->ev_copy, p->copy_stream));
  }
  if (cert) {
    for (int round = 1; round <= p->opts.max_repairs; ++round) {
      CK(cudaMemcpyAsync(p->h_st, p->d_st, sizeof(ItemState) * p->batch, cudaMemcpyDeviceToHost,
                         p->stream));
      CK(cudaStreamSynchronize(p->stream));
      bool all = true;
      for (int64_t i = 0; i < p->batch; ++i)
        if (!p->h_st[i].certified && p->h_st[i].status != FFCZ_ERR_NONFINITE) all = false;
      if (all) break;
      // FP64 repair: Alg. 1 in FP64 from the current e, then re-certify.
      if (host_out) {   // the early copy must finish reading e first
        CK(cudaStreamWaitEvent(p->stream, p->ev_copy, 0));
        recopy = true;
      }
      upload_params(p, eps_s, eps_f, 0, p->opts.max_iters);
      k_set_repairs<<<(unsigned)((p->batch + 255) / 256), 256, 0, p->stream>>>(p->d_st,
                                                                             (int)p->batch, round);
      g_launches++;
      run_loop<double>(p, e, true);
      cert_reset(p);
      certify(p, e, true);
    }
  }
  CK(cudaEventRecord(p->ev2, p->stream));
  CK(cudaEventSynchronize(p->ev2));
  if (host_out) {
    if (recopy) {
      CK(cudaMemcpyAsync(host_out, e, sizeof(float) * p->total, cudaMemcpyDeviceToHost, p->stream));
      ++copies;
    }
    CK(cudaStreamSynchronize(recopy ? p->stream : p->copy_stream));
  }
  float ms = 0.f, ms_c = 0.f;
  CK(cudaEventElapsedTime(&ms, p->ev0, p->ev2));
  CK(cudaEventElapsedTime(&ms_c, p->ev1, p->ev2));
  fill_stats(p, stats, ms, cert ? ms_c : 0.f, cert);
  if (stats)
    for (int64_t i = 0; i < p->batch; ++i) stats[i].host_copies = copies;
  CK(cudaGetLastError());
  return worst_status(p, cert);
}

// ----- backward ---------------------------------------------------------------
__global__ void k_advance(ItemState* st, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) st[i].t += 1;
}
__global__ void k_set_t(ItemState* st, int n, int t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { st[i].t = t; st[i].done = 0; }
}

void advance(ffcz_plan_s* p, ItemState* st) {
  k_advance<<<(unsigned)((p->batch + 255) / 256), 256, 0, p->stream>>>(st, (int)p->batch);
  g_launches++;
}
void set_t(ffcz_plan_s* p, ItemState* st, int t) {
  k_set_t<<<(unsigned)((p->batch + 255) / 256), 256, 0, p->stream>>>(st, (int)p->batch, t);
  g_launches++;
}

// Mask threads per group member of the x pass and of the check pass (the
// words of member gi start at gi x threads x words per thread).
int64_t px_mask_thr(const DevGroup& dg) { return x_words(dg.M, dg.rows, dg.wx) / mask_words_per_thread(dg.M); }
int64_t chk_mask_thr(const DevGroup& dg) {
  return chkw(dg.Nz, dg.ndim == 3 ? dg.Ny : 1, dg.M, dg.wc) / mask_words_per_thread(dg.Nz);
}

// One forward iteration body with mask recording (replay), no decide, for
// every group.  smask / fmask: one step's mask block (group g's words at
// bw_pxoff[g] / bw_chkoff[g]).
void replay_body(ffcz_plan_s* p, LoopBufs B, uint32_t* smask, uint32_t* fmask, float* ckpt, bool do_chk) {
  for (size_t gidx = 0; gidx < p->groups.size(); ++gidx) {
    const DevGroup& dg = p->groups[gidx];
    Args a = make_args<float>(p, dg, B.b0, B.b1, p->d_st);
    a.pred = P_ALL;
    if (dg.ndim == 3) {
      set_tw<float>(a, p->tb, dg.Ny);
      a.sel_in = S_PREV; a.sel_out = S_CUR;
      launch_axis<float, +1>(dg.Ny, dg.wa, a, dg.Nz, dg.M, dg.count, p->stream);
      a.sel_in = S_CUR;
    } else {
      a.sel_in = S_PREV; a.sel_out = S_CUR;
    }
    tabs_x<float>(p, a, dg);
    a.mode = M_CLIP | (smask ? M_RECORD : 0) | (ckpt ? M_CKPT : 0);
    a.mask = smask ? smask + p->bw_pxoff[gidx] : nullptr;
    a.mask_thr = px_mask_thr(dg);
    a.ckpt = ckpt;
    a.ckpt_every = p->bw_m;
    launch_x<float>(XPX, dg.M, dg.wx, a, dg.rows, dg.count, p->stream);
    if (!do_chk) continue;
    a.sel_in = a.sel_out = S_CUR;
    a.mask = nullptr;
    a.ckpt = nullptr;
    if (dg.ndim == 3) {
      set_tw<float>(a, p->tb, dg.Ny);
      a.mode = 0;
      launch_axis<float, -1>(dg.Ny, dg.wa, a, dg.Nz, dg.M, dg.count, p->stream);
    }
    set_tw<float>(a, p->tb, dg.Nz);
    a.mode = M_CLIP | (fmask ? M_RECORD : 0);
    a.mask = fmask ? fmask + p->bw_chkoff[gidx] : nullptr;
    a.mask_thr = chk_mask_thr(dg);
    launch_chk<float>(dg.Nz, dg.wc, a, dg.ndim == 3 ? dg.Ny : 1, dg.M, dg.count, p->stream);
  }
}

void replay_entry(ffcz_plan_s* p, LoopBufs B, float* e0, uint32_t* fmask) {
  for (size_t gidx = 0; gidx < p->groups.size(); ++gidx) {
    const DevGroup& dg = p->groups[gidx];
    Args a = make_args<float>(p, dg, B.b0, B.b1, p->d_st);
    a.pred = P_ALL;
    tabs_x<float>(p, a, dg);
    a.e = e0;
    a.mode = 0;
    launch_x<float>(XFWD, dg.M, dg.wx, a, dg.rows, dg.count, p->stream);
    if (dg.ndim == 3) {
      set_tw<float>(a, p->tb, dg.Ny);
      launch_axis<float, -1>(dg.Ny, dg.wa, a, dg.Nz, dg.M, dg.count, p->stream);
    }
    set_tw<float>(a, p->tb, dg.Nz);
    a.mode = M_CLIP | (fmask ? M_RECORD : 0);
    a.mask = fmask ? fmask + p->bw_chkoff[gidx] : nullptr;
    a.mask_thr = chk_mask_thr(dg);
    launch_chk<float>(dg.Nz, dg.wc, a, dg.ndim == 3 ? dg.Ny : 1, dg.M, dg.count, p->stream);
  }
}

// Plan checks shared by the differentiable entry points.
void bw_check(ffcz_plan_s* p) {
  if (p->opts.pointwise) fail(FFCZ_ERR_INVALID, "backward uses scalar bounds");
  if (p->opts.method != PV_POCS) fail(FFCZ_ERR_UNSUPPORTED, "backward differentiates Alg. 1 (method 0)");
  if (p->opts.K < 1 || p->opts.ckpt_every < 1) fail(FFCZ_ERR_INVALID, "K and ckpt_every must be >= 1");
}

// Workspace of the backward (checkpoints, masks, adjoint buffers), sized
// for the plan's K and ckpt_every: per step one block of x-pass masks and
// one of check-pass masks, the groups' members back to back in each.
void bw_alloc(ffcz_plan_s* p) {
  const int K = p->opts.K, m = p->opts.ckpt_every;
  const int64_t N = p->total;
  const int nseg = (K + m - 1) / m;
  if (p->bw_K != K || p->bw_m != m) {
    p->bw_pxoff.clear();
    p->bw_chkoff.clear();
    int64_t px = 0, ck = 0;
    if (p->ndim == 1) {   // one mask byte per point and per bin k < N, items at their point offsets
      px = ck = (N + 3) / 4;
    } else {
      for (const DevGroup& dg : p->groups) {
        p->bw_pxoff.push_back(px);
        p->bw_chkoff.push_back(ck);
        px += x_words(dg.M, dg.rows, dg.wx) * dg.count;
        ck += chkw(dg.Nz, dg.ndim == 3 ? dg.Ny : 1, dg.M, dg.wc) * dg.count;
      }
    }
    p->px_words = px;
    p->chk_words = ck;
    p->bw_e = (float*)dalloc(p, sizeof(float) * N);
    p->bw_ck = (float*)dalloc(p, sizeof(float) * N * nseg);
    p->bw_smask = (uint32_t*)dalloc(p, sizeof(uint32_t) * p->px_words * m);
    p->bw_fmask = (uint32_t*)dalloc(p, sizeof(uint32_t) * p->chk_words * m);
    if (!p->bw_G[0]) {   // the adjoint's spectra: the plan's spectrum length (1D: P per item)
      p->bw_G[0] = dalloc(p, sizeof(float2) * p->total_c);
      p->bw_G[1] = dalloc(p, sizeof(float2) * p->total_c);
    }
    p->bw_K = K;
    p->bw_m = m;
  }
}

// pre-clip adjoint from the t = 0 checkpoint: a point was clipped exactly
// where the checkpoint differs from e0 (a NaN input included)
__global__ void k_premask_ck(float* g, const float* e0, const float* ck0, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!(ck0[i] == e0[i])) g[i] = 0.f;
}

// 1D items (Bluestein passes): one forward body with mask recording or
// checkpoint writes (replay), and the adjoint's passes.  Masks: one byte per
// point (s) and per bin (f) at the items' point offsets.
void replay_body1(ffcz_plan_s* p, LoopBufs B, uint32_t* smask, uint32_t* fmask, float* ckpt, bool do_chk) {
  for (const DevGroup& dg : p->groups) {
    Args a = make_args<float>(p, dg, B.b0, B.b1, p->d_st);
    a.pred = P_ALL;
    row1_args<float>(p, a, dg, OP1_CONVC);
    a.sel_in = S_PREV; a.sel_out = S_CUR;
    launch_row1<float>(dg.P2, dg.w1r, a, dg.P1, dg.count, p->stream);
    a.sel_in = S_CUR;
    col1_args<float>(p, a, dg, OP1_SCLIP);
    a.mode = M_CLIP | (smask ? M_RECORD : 0) | (ckpt ? M_CKPT : 0);
    a.mask = smask;
    a.ckpt = ckpt;
    a.ckpt_every = p->bw_m;
    launch_col1<float>(dg.P1, dg.w1c, a, dg.P2, dg.count, p->stream);
    if (!do_chk) continue;
    a.mask = nullptr;
    a.ckpt = nullptr;
    row1_args<float>(p, a, dg, OP1_CONV);
    a.mode = 0;
    launch_row1<float>(dg.P2, dg.w1r, a, dg.P1, dg.count, p->stream);
    col1_args<float>(p, a, dg, OP1_FCLIP);
    a.mode = M_CLIP | (fmask ? M_RECORD : 0);
    a.mask = fmask;
    launch_col1<float>(dg.P1, dg.w1c, a, dg.P2, dg.count, p->stream);
  }
}

void replay_entry1(ffcz_plan_s* p, LoopBufs B, float* e0, uint32_t* fmask) {
  for (const DevGroup& dg : p->groups) {
    Args a = make_args<float>(p, dg, B.b0, B.b1, p->d_st);
    a.pred = P_ALL;
    col1_args<float>(p, a, dg, OP1_ENTRY);
    a.e = e0;
    a.mode = 0;
    launch_col1<float>(dg.P1, dg.w1c, a, dg.P2, dg.count, p->stream);
    row1_args<float>(p, a, dg, OP1_CONV);
    launch_row1<float>(dg.P2, dg.w1r, a, dg.P1, dg.count, p->stream);
    col1_args<float>(p, a, dg, OP1_FCLIP);
    a.mode = M_CLIP | (fmask ? M_RECORD : 0);
    a.mask = fmask;
    launch_col1<float>(dg.P1, dg.w1c, a, dg.P2, dg.count, p->stream);
  }
}

// One adjoint step g <- Re(IDFT(M_f DFT(M_s g))) of every 1D item: the
// first takes g from gout (column entry with M_s), the others from the
// previous step's spectrum (row with conj Bt, column with M_s).
void adjoint_step1(ffcz_plan_s* p, LoopBufs GB, const float* gout, uint32_t* sm, uint32_t* fm, bool first) {
  for (const DevGroup& dg : p->groups) {
    Args a = make_args<float>(p, dg, GB.b0, GB.b1, p->d_st2);
    a.pred = P_ALL;
    if (first) {
      col1_args<float>(p, a, dg, OP1_ENTRY);
      a.e = const_cast<float*>(gout);
    } else {
      row1_args<float>(p, a, dg, OP1_CONVC);
      a.sel_in = S_PREV; a.sel_out = S_CUR;
      a.mode = 0;
      launch_row1<float>(dg.P2, dg.w1r, a, dg.P1, dg.count, p->stream);
      a.sel_in = S_CUR;
      col1_args<float>(p, a, dg, OP1_SCLIP);
    }
    a.mode = M_MASK;
    a.mask = sm;
    launch_col1<float>(dg.P1, dg.w1c, a, dg.P2, dg.count, p->stream);
    a.sel_in = a.sel_out = S_CUR;
    row1_args<float>(p, a, dg, OP1_CONV);
    a.mode = 0;
    a.mask = nullptr;
    launch_row1<float>(dg.P2, dg.w1r, a, dg.P1, dg.count, p->stream);
    col1_args<float>(p, a, dg, OP1_FCLIP);
    a.mode = M_MASK;
    a.mask = fm;
    launch_col1<float>(dg.P1, dg.w1c, a, dg.P2, dg.count, p->stream);
  }
}

// The segments of the 1D backward (after the forward's checkpoints).
ffcz_status backward1_tail(ffcz_plan_s* p, const float* e0, const float* gout, float* gin, const float* ck,
                           const float* ckpt_in, LoopBufs B, LoopBufs GB) {
  const int K = p->opts.K, m = p->opts.ckpt_every;
  const int64_t N = p->total;
  const int nseg = (K + m - 1) / m;
  // with the masks the forward kept (opts.keep_masks) no segment is replayed
  const bool kept = ckpt_in && p->opts.keep_masks && p->km_valid && p->km_K == K;
  set_t(p, p->d_st2, 0);
  bool first = true;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int t0 = seg * m, t1 = std::min(K, t0 + m);
    if (!kept) {
      set_t(p, p->d_st, t0);
      replay_entry1(p, B, const_cast<float*>(ck) + (int64_t)seg * N, p->bw_fmask);
      for (int b = t0 + 1; b <= t1; ++b) {
        advance(p, p->d_st);
        replay_body1(p, B, p->bw_smask + (int64_t)(b - 1 - t0) * p->px_words,
                     b < t1 ? p->bw_fmask + (int64_t)(b - t0) * p->chk_words : nullptr, nullptr, b < t1);
      }
    }
    for (int t = t1 - 1; t >= t0; --t) {
      if (!first) advance(p, p->d_st2);
      uint32_t* sm = kept ? p->km_s + (int64_t)(t + 1) * p->px_words : p->bw_smask + (int64_t)(t - t0) * p->px_words;
      uint32_t* fm = kept ? p->km_f + (int64_t)t * p->chk_words : p->bw_fmask + (int64_t)(t - t0) * p->chk_words;
      adjoint_step1(p, GB, gout, sm, fm, first);
      first = false;
    }
  }
  // exit: x = Re(b c) / (P N) of the last step's spectrum, no clip
  advance(p, p->d_st2);
  for (const DevGroup& dg : p->groups) {
    Args a = make_args<float>(p, dg, GB.b0, GB.b1, p->d_st2);
    a.pred = P_ALL;
    row1_args<float>(p, a, dg, OP1_CONVC);
    a.sel_in = S_PREV; a.sel_out = S_CUR;
    launch_row1<float>(dg.P2, dg.w1r, a, dg.P1, dg.count, p->stream);
    a.sel_in = S_CUR;
    col1_args<float>(p, a, dg, OP1_EXIT);
    a.e = gin;
    a.mode = 0;
    launch_col1<float>(dg.P1, dg.w1c, a, dg.P2, dg.count, p->stream);
  }
  if (ckpt_in) {
    k_premask_ck<<<1184, 256, 0, p->stream>>>(gin, e0, ckpt_in, N);
    g_launches++;
  } else {
    for (int64_t i = 0; i < p->batch; ++i) {
      const int64_t n = p->h_prm[i].n;
      k_premask<<<(unsigned)std::min<int64_t>(1184, (n + 255) / 256), 256, 0, p->stream>>>(
          gin + p->eoff[i], e0 + p->eoff[i], p->d_prm, p->d_st, (int)i, n);
      g_launches++;
    }
  }
  CK(cudaStreamSynchronize(p->stream));
  CK(cudaGetLastError());
  return FFCZ_OK;
}

// ckpt_in: checkpoints written by ffcz_correct_ckpt (null: the forward is run
// again here to take them).  Every item runs exactly K steps, so all items
// (any number of shape groups) go through the segments together.
ffcz_status backward_impl(ffcz_plan_s* p, const float* e0, const float* gout, float* gin,
                          const double* eps_s, const double* eps_f, const float* ckpt_in = nullptr) {
  bw_check(p);
  if (!e0 || !gout || !gin || !eps_s || !eps_f) fail(FFCZ_ERR_INVALID, "null pointer argument");
  const int K = p->opts.K, m = p->opts.ckpt_every;
  CK(cudaSetDevice(p->device));
  ProfOn prof_on(p);
  const int64_t N = p->total;
  const int nseg = (K + m - 1) / m;
  bw_alloc(p);
  upload_params(p, eps_s, eps_f, K, K);
  LoopBufs B{p->B32[0], p->B32[1]};
  LoopBufs GB{p->bw_G[0], p->bw_G[1]};
  // Forward with checkpoints of e_t at t = 0, m, 2m, ... (t < K).
  CK(cudaMemsetAsync(p->d_nactive, 0, sizeof(int), p->stream));
  k_init<<<(unsigned)((p->batch + 255) / 256), 256, 0, p->stream>>>(p->d_st, (int)p->batch, 0, p->d_nactive);
  g_launches++;
  const float* ck = ckpt_in ? ckpt_in : p->bw_ck;
  if (!ckpt_in) {
    CK(cudaMemcpyAsync(p->bw_e, e0, sizeof(float) * N, cudaMemcpyDeviceToDevice, p->stream));
    // entry with A3 pre-clip on the working copy
    entry<float>(p, B, p->bw_e, true, p->stream);
    CK(cudaMemcpyAsync(p->bw_ck, p->bw_e, sizeof(float) * N, cudaMemcpyDeviceToDevice, p->stream));
    const int last_ck = (nseg - 1) * m;
    for (int t = 1; t <= last_ck; ++t) {
      // k_decide after entry set t = 1 (forced iterations never stop early)
      if (p->ndim == 1) replay_body1(p, B, nullptr, nullptr, p->bw_ck, t < last_ck);
      else replay_body(p, B, nullptr, nullptr, p->bw_ck, t < last_ck);
      if (t < last_ck) advance(p, p->d_st);
    }
  }
  if (p->ndim == 1) return backward1_tail(p, e0, gout, gin, ck, ckpt_in, B, GB);
  // Adjoint, segment by segment from the last.  With the masks the forward
  // kept (opts.keep_masks), no segment is replayed: step t takes the x-pass
  // masks of step t + 1 and the check-pass masks of check t.
  const bool kept = ckpt_in && p->opts.keep_masks && p->km_valid && p->km_K == K;
  set_t(p, p->d_st2, 0);
  bool first = true;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int t0 = seg * m, t1 = std::min(K, t0 + m);
    if (!kept) {
      // replay the segment from its checkpoint, recording masks of steps t0..t1-1
      set_t(p, p->d_st, t0);
      replay_entry(p, B, const_cast<float*>(ck) + (int64_t)seg * N, p->bw_fmask);
      for (int b = t0 + 1; b <= t1; ++b) {
        advance(p, p->d_st);
        replay_body(p, B, p->bw_smask + (int64_t)(b - 1 - t0) * p->px_words,
                    b < t1 ? p->bw_fmask + (int64_t)(b - t0) * p->chk_words : nullptr, nullptr, b < t1);
      }
    }
    for (int t = t1 - 1; t >= t0; --t) {
      uint32_t* sm = kept ? p->km_s + (int64_t)(t + 1) * p->px_words : p->bw_smask + (int64_t)(t - t0) * p->px_words;
      uint32_t* fm = kept ? p->km_f + (int64_t)t * p->chk_words : p->bw_fmask + (int64_t)(t - t0) * p->chk_words;
      if (!first) advance(p, p->d_st2);
      for (size_t gidx = 0; gidx < p->groups.size(); ++gidx) {
        const DevGroup& dg = p->groups[gidx];
        Args a = make_args<float>(p, dg, GB.b0, GB.b1, p->d_st2);
        a.pred = P_ALL;
        a.mask_thr = px_mask_thr(dg);
        if (first) {
          tabs_x<float>(p, a, dg);
          a.ein = gout;
          a.e = const_cast<float*>(gout);
          a.mask = sm + p->bw_pxoff[gidx];
          a.mode = M_MASK;
          launch_x<float>(XFWD, dg.M, dg.wx, a, dg.rows, dg.count, p->stream);
        } else {
          if (dg.ndim == 3) {
            set_tw<float>(a, p->tb, dg.Ny);
            a.sel_in = S_PREV; a.sel_out = S_CUR;
            launch_axis<float, +1>(dg.Ny, dg.wa, a, dg.Nz, dg.M, dg.count, p->stream);
            a.sel_in = S_CUR;
          } else {
            a.sel_in = S_PREV; a.sel_out = S_CUR;
          }
          tabs_x<float>(p, a, dg);
          a.mask = sm + p->bw_pxoff[gidx];
          a.mode = M_MASK;
          launch_x<float>(XPX, dg.M, dg.wx, a, dg.rows, dg.count, p->stream);
        }
        a.sel_in = a.sel_out = S_CUR;
        if (dg.ndim == 3) {
          set_tw<float>(a, p->tb, dg.Ny);
          a.mode = 0;
          a.mask = nullptr;
          launch_axis<float, -1>(dg.Ny, dg.wa, a, dg.Nz, dg.M, dg.count, p->stream);
        }
        set_tw<float>(a, p->tb, dg.Nz);
        a.mode = M_MASK;
        a.mask = fm + p->bw_chkoff[gidx];
        a.mask_thr = chk_mask_thr(dg);
        launch_chk<float>(dg.Nz, dg.wc, a, dg.ndim == 3 ? dg.Ny : 1, dg.M, dg.count, p->stream);
      }
      first = false;
    }
  }
  // exit: inverse of the last step's spectrum, no clip
  advance(p, p->d_st2);
  for (const DevGroup& dg : p->groups) {
    Args a = make_args<float>(p, dg, GB.b0, GB.b1, p->d_st2);
    a.pred = P_ALL;
    a.e = gin;
    if (dg.ndim == 3) {
      set_tw<float>(a, p->tb, dg.Ny);
      a.sel_in = S_PREV; a.sel_out = S_CUR;
      launch_axis<float, +1>(dg.Ny, dg.wa, a, dg.Nz, dg.M, dg.count, p->stream);
      a.sel_in = S_CUR;
    } else {
      a.sel_in = S_PREV;
    }
    tabs_x<float>(p, a, dg);
    a.mode = 0;
    launch_x<float>(XEXIT, dg.M, dg.wx, a, dg.rows, dg.count, p->stream);
  }
  if (ckpt_in) {
    k_premask_ck<<<1184, 256, 0, p->stream>>>(gin, e0, ckpt_in, N);
    g_launches++;
  } else {
    for (int64_t i = 0; i < p->batch; ++i) {
      const int64_t n = p->h_prm[i].n;
      k_premask<<<(unsigned)std::min<int64_t>(1184, (n + 255) / 256), 256, 0, p->stream>>>(
          gin + p->eoff[i], e0 + p->eoff[i], p->d_prm, p->d_st, (int)i, n);
      g_launches++;
    }
  }
  CK(cudaStreamSynchronize(p->stream));
  CK(cudaGetLastError());
  return FFCZ_OK;
}

}  // namespace

namespace {

// ----- tile-width tuner ----------------------------------------------------------
// For every group and float32 pass kind, time the variants of the pass
// (strided passes: 4- and 8-pencil tiles and, for lengths >= 256, the
// persistent TMA-fed kernel, code -8; contiguous passes: tiles of one and two
// warps) on the plan's own buffers (three launches each after one warm-up,
// CUDA events) and keep the fastest.  Results can be cached in a text file named by
// FFCZ_TUNE_CACHE (lines "key width"); FFCZ_TUNE=0 keeps the defaults.
std::map<std::string, int>& tune_table() {
  static std::map<std::string, int> t;
  return t;
}
std::mutex& tune_mu() {
  static std::mutex m;
  return m;
}
void tune_load() {
  static bool loaded = false;
  if (loaded) return;
  loaded = true;
  const char* f = getenv("FFCZ_TUNE_CACHE");
  if (!f) return;
  FILE* fp = fopen(f, "r");
  if (!fp) return;
  char key[256];
  int w;
  while (fscanf(fp, "%255s %d", key, &w) == 2) tune_table()[key] = w;
  fclose(fp);
}
void tune_store(const std::string& key, int w) {
  tune_table()[key] = w;
  const char* f = getenv("FFCZ_TUNE_CACHE");
  if (!f) return;
  FILE* fp = fopen(f, "a");
  if (!fp) return;
  fprintf(fp, "%s %d\n", key.c_str(), w);
  fclose(fp);
}

template <typename F>
float time_launches(ffcz_plan_s* p, F&& f) {
  f();   // warm-up (and module load)
  CK(cudaEventRecord(p->ev0, p->stream));
  for (int i = 0; i < 3; ++i) f();
  CK(cudaEventRecord(p->ev1, p->stream));
  CK(cudaEventSynchronize(p->ev1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
  return ms;
}

// FFCZ_TUNE_FORCE="kind=w,..." (kinds px, axis, chk, col1, row1; w a tile
// width or "tma" for the persistent copy-engine-fed variant) fixes a pass's
// variant for plans created while it is set, if w is one of its candidates.
int forced_width(const std::string& key, const std::vector<int>& cand) {
  const char* f = getenv("FFCZ_TUNE_FORCE");
  if (!f) return 0;
  const std::string kind = key.substr(0, key.find('_'));
  std::string spec(f);
  size_t pos = 0;
  while (pos < spec.size()) {
    size_t end = spec.find(',', pos);
    if (end == std::string::npos) end = spec.size();
    const std::string item = spec.substr(pos, end - pos);
    const size_t eq = item.find('=');
    if (eq != std::string::npos && item.substr(0, eq) == kind) {
      const std::string val = item.substr(eq + 1);
      if (val == "tma") {   // the persistent copy-engine-fed variant (negative code)
        for (int c : cand)
          if (c < 0) return c;
        return 0;
      }
      const int w = atoi(val.c_str());
      if (std::find(cand.begin(), cand.end(), w) != cand.end()) return w;
    }
    pos = end + 1;
  }
  return 0;
}

thread_local bool g_no_tune = false;   // FFCZ_TUNE=0: keep the defaults

template <typename F>
int pick_width(ffcz_plan_s* p, const std::string& key, int dflt, std::vector<int> cand, F&& run_w) {
  if (const int w = forced_width(key, cand)) return w;
  if (g_no_tune) return dflt;
  {
    std::lock_guard<std::mutex> lk(tune_mu());
    tune_load();
    auto it = tune_table().find(key);
    if (it != tune_table().end() && std::find(cand.begin(), cand.end(), it->second) != cand.end())
      return it->second;
  }
  int best = cand[0];
  float tbest = 0.f;
  for (size_t i = 0; i < cand.size(); ++i) {
    const float t = time_launches(p, [&] { run_w(cand[i]); });
    if (i == 0 || t < tbest) { tbest = t; best = cand[i]; }
  }
  std::lock_guard<std::mutex> lk(tune_mu());
  tune_store(key, best);
  return best;
}

// FFCZ_TUNE_FORCE="...,split=0" (or 1) fixes the radix split of every
// tuned pass whose length allows both; returns -1 when not forced.
int forced_split() {
  const char* f = getenv("FFCZ_TUNE_FORCE");
  if (!f) return -1;
  const std::string spec(f);
  const size_t pos = spec.find("split=");
  if (pos == std::string::npos) return -1;
  return spec[pos + 6] == '1' ? 1 : 0;
}

// A pass's variant: tile width and, where the length allows both, radix
// split.  The split of a pass kind and length is ONE decision per process
// (and per tune cache): the first plan that needs it times every candidate
// of both splits and the winner's split is kept; later groups of that kind
// and length tune their tile widths within it.  Tile widths and the
// copy-engine-fed kernels only regroup the same arithmetic, the split changes
// its order, so this keeps every plan that shares a length on the same
// arithmetic (a batch and its single items agree bit for bit).
template <typename F>
int pick_variant(ffcz_plan_s* p, const std::string& kind, const std::string& key, int L, int dflt,
                 const std::vector<int>& cand0, F&& run_w) {
  std::vector<int> both = cand0;
  if (split_ok(L, 1))
    for (int c : cand0)
      if (c > 0) both.push_back(c | kSplit);
  if (const int w = forced_width(key, both)) return w;
  if (!split_ok(L, 1)) return pick_width(p, key, dflt, cand0, run_w);
  int S = forced_split();
  const std::string skey = "split_" + kind + "_L" + std::to_string(L);
  if (S < 0 && !g_no_tune) {
    std::lock_guard<std::mutex> lk(tune_mu());
    tune_load();
    auto it = tune_table().find(skey);
    if (it != tune_table().end()) S = it->second ? 1 : 0;
  }
  if (g_no_tune && S < 0) S = 0;
  if (S == 0) return pick_width(p, key + "_s0", dflt, cand0, run_w);
  if (S == 1) {
    std::vector<int> c1;
    for (int c : cand0)
      if (c > 0) c1.push_back(c | kSplit);
    return pick_width(p, key + "_s1", c1[0], c1, run_w);
  }
  const int best = pick_width(p, key + "_sx", dflt, both, run_w);
  std::lock_guard<std::mutex> lk(tune_mu());
  tune_store(skey, (best > 0 && (best & kSplit)) ? 1 : 0);
  return best;
}

// FFCZ_TUNE_FORCE="...,multi=1" (or 0) fixes the form of every loop pass
// of multi-group plans; returns -1 when not forced.
int forced_multi() {
  const char* f = getenv("FFCZ_TUNE_FORCE");
  if (!f) return -1;
  const std::string spec(f);
  const size_t pos = spec.find("multi=");
  if (pos == std::string::npos) return -1;
  return spec[pos + 6] == '1' ? 1 : 0;
}

// For plans of several shape groups: time each pass kind of the float32
// loop over all groups, as separate launches (each group's tuned variant)
// and as one multi-group launch, and keep the faster form per kind.
void tune_multi(ffcz_plan_s* p) {
  const int ng = (int)p->groups.size();
  const int forced = forced_multi();
  cudaStream_t s = p->stream;
  std::string gkey = "multi_d" + std::to_string(p->ndim);
  for (const auto& dg : p->groups) {
    char b[96];
    snprintf(b, sizeof b, "_%dx%dx%dx%d_%d", dg.Nz, dg.Ny, dg.Nx, dg.P1, dg.count);
    gkey += b;
  }
  for (int k = 0; k < MK_N; ++k) {
    if (p->mp[k].n == 0) continue;
    // the multi-group units run the default radix split
    bool split_any = false;
    for (const auto& dg : p->groups) {
      const int w = k == MK_PX ? dg.wx : (k == MK_YINV || k == MK_YFWD) ? dg.wa : k == MK_CHK ? dg.wc : 0;
      split_any |= w > 0 && (w & kSplit);
    }
    if (split_any) { p->multi_use[k] = false; continue; }
    if (forced >= 0) { p->multi_use[k] = forced == 1; continue; }
    if (g_no_tune) continue;
    const std::string key = gkey + "_" + multi_name(k);
    {
      std::lock_guard<std::mutex> lk(tune_mu());
      tune_load();
      auto it = tune_table().find(key);
      if (it != tune_table().end()) { p->multi_use[k] = it->second == 1; continue; }
    }
    std::vector<Args> args(ng);
    for (int g = 0; g < ng; ++g) {
      const DevGroup& dg = p->groups[g];
      Args a = make_args<float>(p, dg, p->B32[0], p->B32[1], p->d_st);
      a.pred = P_ALL;
      if (k == MK_PX) { tabs_x<float>(p, a, dg); a.mode = M_CLIP; }
      else if (k == MK_YINV || k == MK_YFWD) set_tw<float>(a, p->tb, dg.Ny);
      else if (k == MK_CHK) { set_tw<float>(a, p->tb, dg.Nz); a.mode = M_CLIP; }
      else if (k == MK_COL1) { col1_args<float>(p, a, dg, OP1_SCLIP); a.mode = M_CLIP; }
      else row1_args<float>(p, a, dg, OP1_CONV);
      args[g] = a;
    }
    const float t_sep = time_launches(p, [&] {
      for (int g = 0; g < ng; ++g) {
        const DevGroup& dg = p->groups[g];
        const Args& a = args[g];
        switch (k) {
          case MK_PX: launch_x<float>(XPX, dg.M, dg.wx, a, dg.rows, dg.count, s); break;
          case MK_YINV: launch_axis<float, +1>(dg.Ny, dg.wa, a, dg.Nz, dg.M, dg.count, s); break;
          case MK_YFWD: launch_axis<float, -1>(dg.Ny, dg.wa, a, dg.Nz, dg.M, dg.count, s); break;
          case MK_CHK: launch_chk<float>(dg.Nz, dg.wc, a, dg.ndim == 3 ? dg.Ny : 1, dg.M, dg.count, s); break;
          case MK_COL1: launch_col1<float>(dg.P1, dg.w1c, a, dg.P2, dg.count, s); break;
          default: launch_row1<float>(dg.P2, dg.w1r, a, dg.P1, dg.count, s); break;
        }
      }
    });
    const float t_multi = time_launches(p, [&] { multi_launch<float>(p, k, args, s, true); });
    p->multi_use[k] = t_multi < t_sep;
    std::lock_guard<std::mutex> lk(tune_mu());
    tune_store(key, p->multi_use[k] ? 1 : 0);
  }
}

void tune(ffcz_plan_s* p) {
  const char* env = getenv("FFCZ_TUNE");
  g_no_tune = env && env[0] == '0';
  if (g_no_tune && !getenv("FFCZ_TUNE_FORCE")) return;
  cudaStream_t s = p->stream;
  for (auto& dg : p->groups) {
    char base[160];
    snprintf(base, sizeof base, "d%d_z%d_y%d_x%d_n%d_c%d_pw%d", dg.ndim, dg.Nz, dg.Ny, dg.Nx, dg.P1,
             dg.count, p->opts.pointwise ? 1 : 0);
    Args a = make_args<float>(p, dg, p->B32[0], p->B32[1], p->d_st);
    a.pred = P_ALL;
    if (dg.ndim == 1) {
      dg.w1c = pick_width(p, std::string("col1_") + base, dg.w1c, {4, 8}, [&](int w) {
        Args b = a;
        col1_args<float>(p, b, dg, OP1_SCLIP);
        b.mode = 0;
        launch_col1<float>(dg.P1, w, b, dg.P2, dg.count, s);
      });
      dg.w1r = pick_width(p, std::string("row1_") + base, dg.w1r, {row_w1(dg.P2), row_w2(dg.P2)}, [&](int w) {
        Args b = a;
        row1_args<float>(p, b, dg, OP1_FWD);
        launch_row1<float>(dg.P2, w, b, dg.P1, dg.count, s);
      });
      continue;
    }
    // candidates: tile widths, the persistent copy-engine-fed kernel, and
    // (odd log2 of the length) the swapped radix split of the plain kernel
    dg.wx = pick_variant(p, "px", std::string("px_") + base, dg.M, dg.wx,
                         {row_w1(dg.M), row_w2(dg.M), -row_w1(dg.M)}, [&](int w) {
      Args b = a;
      tabs_x<float>(p, b, dg);
      b.mode = 0;
      launch_x<float>(XPX, dg.M, w, b, dg.rows, dg.count, s);
    });
    if (dg.ndim == 3)
      dg.wa = pick_variant(p, "axis", std::string("axis_") + base, dg.Ny, dg.wa,
                           dg.tm_axis ? std::vector<int>{4, 8, -8} : std::vector<int>{4, 8}, [&](int w) {
        Args b = a;
        set_tw<float>(b, p->tb, dg.Ny);
        launch_axis<float, -1>(dg.Ny, w, b, dg.Nz, dg.M, dg.count, s);
      });
    dg.wc = pick_variant(p, "chk", std::string("chk_") + base, dg.Nz, dg.wc,
                         dg.tm_chk ? std::vector<int>{4, 8, -8} : std::vector<int>{4, 8}, [&](int w) {
      Args b = a;
      set_tw<float>(b, p->tb, dg.Nz);
      b.mode = 0;
      launch_chk<float>(dg.Nz, w, b, dg.ndim == 3 ? dg.Ny : 1, dg.M, dg.count, s);
    });
  }
  tune_multi(p);
  CK(cudaMemsetAsync(p->d_st, 0, sizeof(ItemState) * p->batch, s));
  CK(cudaMemcpyAsync(p->h_err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  check_dev_err(p);
}

}  // namespace

namespace {

// ----- FP64 pipe peak (measurement support, not part of the method) ---------
// Every thread runs kFpChains independent dependency chains of FP64 FMAs
// (kind 0) or adds (kind 1), enough to cover the pipe's latency, so the
// FP64 issue rate alone bounds the kernel.  The chains' sum is written only
// when it equals a value it never reaches; the compiler cannot know that, so
// no chain is removed.
constexpr int kFpChains = 8;
__global__ void __launch_bounds__(256) k_fp64_peak(double* out, int iters, int kind, double m, double c) {
  double a[kFpChains];
#pragma unroll
  for (int i = 0; i < kFpChains; ++i) a[i] = 1e-3 * threadIdx.x + i;
  if (kind == 0) {
#pragma unroll 4
    for (int t = 0; t < iters; ++t)
#pragma unroll
      for (int i = 0; i < kFpChains; ++i) a[i] = fma(a[i], m, c);
  } else {
#pragma unroll 4
    for (int t = 0; t < iters; ++t)
#pragma unroll
      for (int i = 0; i < kFpChains; ++i) a[i] = a[i] + c;
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kFpChains; ++i) s += a[i];
  if (s == -1.0) out[0] = s;
}

}  // namespace

// Lets the library's other translation unit report a detail message through
// ffcz_last_error() (not exported).
__attribute__((visibility("hidden"))) void ffcz_set_last_error(const char* msg) {
  g_err = msg ? msg : "";
}

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

void ffcz_default_opts(ffcz_opts* o) {
  if (!o) return;
  o->max_iters = 10000;
  o->min_iters = 0;
  o->shrink = 1.0 / 65536.0;
  o->precision = 32;
  o->certify = 1;
  o->max_repairs = 2;
  o->K = 50;
  o->ckpt_every = 10;
  o->chunk = 16;
  o->use_graph = 2;
  o->count_active = 1;
  o->edits = 0;
  o->pointwise = 0;
  o->method = 0;
  o->keep_masks = 0;
}

ffcz_status ffcz_plan(ffcz_plan_t* out, int ndim, const int64_t* shapes, int64_t batch,
                      const ffcz_opts* opts, void* cuda_stream) {
  return guarded([&]() -> ffcz_status {
    if (!out) fail(FFCZ_ERR_INVALID, "out is null");
    *out = nullptr;
    if (!shapes) fail(FFCZ_ERR_INVALID, "shapes is null");
    if (ndim < 1 || ndim > 3) fail(FFCZ_ERR_INVALID, "ndim must be 1..3");
    if (batch < 1 || batch > 65535) fail(FFCZ_ERR_INVALID, "batch must be in [1, 65535]");
    ffcz_opts o;
    ffcz_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != 32 && o.precision != 64) fail(FFCZ_ERR_INVALID, "precision must be 32 or 64");
    if (!(o.shrink >= 0.0 && o.shrink < 0.5)) fail(FFCZ_ERR_INVALID, "shrink must be in [0, 0.5)");
    if (o.max_iters < 0 || o.min_iters < 0) fail(FFCZ_ERR_INVALID, "iteration limits must be >= 0");
    if (o.method < PV_POCS || o.method > PV_ADMM) fail(FFCZ_ERR_INVALID, "method must be 0..3");
    if (o.keep_masks != 0 && o.keep_masks != 1) fail(FFCZ_ERR_INVALID, "keep_masks must be 0 or 1");
    if (o.method != PV_POCS && (o.edits || o.pointwise || o.precision != 32))
      fail(FFCZ_ERR_UNSUPPORTED, "projection variants run float32 loops without edits or pointwise bounds");
    for (int64_t i = 0; i < batch; ++i) {
      if (ndim == 1) {
        const int64_t n = shapes[i];
        if (n < 32 || n > (1 << 19))
          fail(FFCZ_ERR_UNSUPPORTED, "1D lengths must be in [32, 524288]");
        continue;
      }
      for (int d = 0; d < ndim; ++d) {
        const int64_t n = shapes[i * ndim + d];
        const bool last = d == ndim - 1;
        if (!is_pow2(n) || n < (last ? 16 : 8) || n > (last ? 2048 : 1024))
          fail(FFCZ_ERR_UNSUPPORTED, "axis lengths must be powers of two in [8, 1024] "
                                     "([16, 2048] for the last axis)");
      }
    }
    std::unique_ptr<ffcz_plan_s, void (*)(ffcz_plan_s*)> p(new ffcz_plan_s, free_plan);
    p->ndim = ndim;
    p->batch = batch;
    p->shapes.assign(shapes, shapes + batch * ndim);
    p->opts = o;
    p->stream = (cudaStream_t)cuda_stream;
    CK(cudaGetDevice(&p->device));
    CK(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
    g_num_sms = p->num_sms;
    g_num_sms_x = p->num_sms;
    p->eoff.resize(batch);
    std::vector<int64_t> soff_c(batch);
    int64_t off = 0, offc = 0;
    // group key: the shape (2D/3D) or the Bluestein split (P1, P2) (1D)
    std::map<std::vector<int64_t>, std::vector<int>> bys;
    for (int64_t i = 0; i < batch; ++i) {
      std::vector<int64_t> sh(shapes + i * ndim, shapes + (i + 1) * ndim);
      int64_t n = 1;
      for (auto v : sh) n *= v;
      p->eoff[i] = off;
      soff_c[i] = offc;
      off += n;
      if (ndim == 1) {
        const int64_t P = p1d_len(n);
        const int lg = ilog2((int)P);
        const int64_t P1 = (int64_t)1 << (lg / 2);
        offc += P;
        bys[{P1, P / P1}].push_back((int)i);
      } else {
        offc += n / 2;
        bys[sh].push_back((int)i);
      }
    }
    p->total = off;
    p->total_c = offc;
    CK(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    CK(cudaEventCreate(&p->ev0));
    CK(cudaEventCreate(&p->ev1));
    CK(cudaEventCreate(&p->ev2));
    // twiddle tables: stage factors for L = 8..1024, R2C factors for Nx = 16..2048
    for (int pw = 3; pw <= 10; ++pw) {
      const int L = 1 << pw;
      auto t32 = stage_table_rt<float>(L);
      auto t64 = stage_table_rt<double>(L);
      p->tb.f32[pw] = dalloc(p.get(), sizeof(float2) * t32.size());
      p->tb.f64[pw] = dalloc(p.get(), sizeof(double2) * t64.size());
      CK(cudaMemcpy(p->tb.f32[pw], t32.data(), sizeof(float2) * t32.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(p->tb.f64[pw], t64.data(), sizeof(double2) * t64.size(), cudaMemcpyHostToDevice));
      if (split_ok(L, 1)) {
        auto s32 = stage_table_rt<float>(L, 1);
        auto s64 = stage_table_rt<double>(L, 1);
        p->tb.f32s[pw] = dalloc(p.get(), sizeof(float2) * s32.size());
        p->tb.f64s[pw] = dalloc(p.get(), sizeof(double2) * s64.size());
        CK(cudaMemcpy(p->tb.f32s[pw], s32.data(), sizeof(float2) * s32.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(p->tb.f64s[pw], s64.data(), sizeof(double2) * s64.size(), cudaMemcpyHostToDevice));
      }
    }
    for (int pw = 4; pw <= 11; ++pw) {
      const int Nx = 1 << pw;
      auto t32 = r2c_table<float>(Nx);
      auto t64 = r2c_table<double>(Nx);
      p->tb.r32[pw] = dalloc(p.get(), sizeof(float2) * t32.size());
      p->tb.r64[pw] = dalloc(p.get(), sizeof(double2) * t64.size());
      CK(cudaMemcpy(p->tb.r32[pw], t32.data(), sizeof(float2) * t32.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(p->tb.r64[pw], t64.data(), sizeof(double2) * t64.size(), cudaMemcpyHostToDevice));
    }
    for (auto& kv : bys) {
      const auto& sh = kv.first;
      const auto& ids = kv.second;
      DevGroup dg{};
      dg.ndim = ndim;
      dg.count = (int)ids.size();
      if (ndim == 1) {
        dg.P1 = (int)sh[0];
        dg.P2 = (int)sh[1];
        dg.Nz = dg.P1;           // rows of the [P1][P2] array
        dg.M = dg.P2;            // row length
        dg.Ny = 1;
        dg.Nx = 2 * dg.P2;
        dg.n = (int64_t)dg.P1 * dg.P2;
        dg.rows = dg.P1;
        const int P = dg.P1 * dg.P2;
        std::vector<float2> t32(P);
        std::vector<double2> t64(P);
        for (int m = 0; m < P; ++m) {
          const double2 r = root<double>(m, P);
          t64[m] = r;
          const float2 f = root<float>(m, P);
          t32[m] = f;
        }
        void* d32 = dalloc(p.get(), sizeof(float2) * P);
        void* d64 = dalloc(p.get(), sizeof(double2) * P);
        CK(cudaMemcpy(d32, t32.data(), sizeof(float2) * P, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d64, t64.data(), sizeof(double2) * P, cudaMemcpyHostToDevice));
        dg.twp32 = d32;
        dg.twp64 = d64;
      } else {
        dg.Nx = (int)sh[ndim - 1];
        dg.M = dg.Nx / 2;
        dg.Nz = (int)sh[0];
        dg.Ny = ndim == 3 ? (int)sh[1] : 1;
        dg.n = 1;
        for (auto v : sh) dg.n *= v;
        dg.rows = dg.n / dg.Nx;
      }
      dg.wx = row_w1(dg.M);
      dg.w1r = row_w1(dg.M);
      std::vector<int32_t> it(ids.begin(), ids.end());
      std::vector<int64_t> eo, so;
      for (int id : ids) { eo.push_back(p->eoff[id]); so.push_back(soff_c[id]); }
      {
        // each member's offset in the half spectra of a real-input FFT,
        // items back to back (1D items: N/2 + 1 bins)
        std::vector<int64_t> co;
        int64_t acc = 0;
        std::vector<int64_t> canon(batch);
        for (int64_t i = 0; i < batch; ++i) {
          canon[i] = acc;
          int64_t nb = 1;
          for (int d = 0; d < ndim - 1; ++d) nb *= shapes[i * ndim + d];
          acc += nb * (shapes[i * ndim + ndim - 1] / 2 + 1);
        }
        for (int id : ids) co.push_back(canon[id]);
        int64_t* d_co = (int64_t*)dalloc(p.get(), sizeof(int64_t) * co.size());
        CK(cudaMemcpy(d_co, co.data(), sizeof(int64_t) * co.size(), cudaMemcpyHostToDevice));
        dg.d_canon = d_co;
        dg.g.coff = d_co;
      }
      if (ndim > 1) {
        // x-row offsets (rows = points / Nx) of every item, for per-row tables
        std::vector<int64_t> rowoff(batch), ro;
        int64_t racc = 0;
        for (int64_t i = 0; i < batch; ++i) {
          rowoff[i] = racc;
          int64_t r = 1;
          for (int d = 0; d < ndim - 1; ++d) r *= shapes[i * ndim + d];
          racc += r;
        }
        p->total_rows = racc;
        for (int id : ids) ro.push_back(rowoff[id]);
        int64_t* d_ro = (int64_t*)dalloc(p.get(), sizeof(int64_t) * ro.size());
        CK(cudaMemcpy(d_ro, ro.data(), sizeof(int64_t) * ro.size(), cudaMemcpyHostToDevice));
        dg.g.roff = d_ro;
      }
      int32_t* d_it = (int32_t*)dalloc(p.get(), sizeof(int32_t) * it.size());
      int64_t* d_eo = (int64_t*)dalloc(p.get(), sizeof(int64_t) * eo.size());
      int64_t* d_so = (int64_t*)dalloc(p.get(), sizeof(int64_t) * so.size());
      CK(cudaMemcpy(d_it, it.data(), sizeof(int32_t) * it.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_eo, eo.data(), sizeof(int64_t) * eo.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(d_so, so.data(), sizeof(int64_t) * so.size(), cudaMemcpyHostToDevice));
      dg.g.ndim = ndim;
      dg.g.Nz = dg.Nz;
      dg.g.Nmid = dg.Ny;
      dg.g.M = dg.M;
      dg.g.rows = dg.rows;
      dg.g.item = d_it;
      dg.g.eoff = d_eo;
      dg.g.soff = d_so;
      dg.h_soff = so;
      p->groups.push_back(dg);
    }
    if (ndim == 1) {
      // groups of the N/2-point certification passes (even N >= 64): the
      // Bluestein length is P/2, split like any other; members keep their
      // point, spectrum and half-spectrum offsets
      std::map<std::pair<int64_t, int64_t>, std::vector<int>> hby;
      std::vector<int64_t> canon(batch);
      int64_t acc = 0;
      for (int64_t i = 0; i < batch; ++i) {
        canon[i] = acc;
        acc += shapes[i] / 2 + 1;
        if (!half_cert_ok(shapes[i])) continue;
        const int64_t Ph = p1d_len(shapes[i] / 2);
        const int64_t P1 = (int64_t)1 << (ilog2((int)Ph) / 2);
        hby[{P1, Ph / P1}].push_back((int)i);
      }
      for (auto& kv : hby) {
        const auto& ids = kv.second;
        DevGroup hg{};
        hg.ndim = 1;
        hg.count = (int)ids.size();
        hg.P1 = (int)kv.first.first;
        hg.P2 = (int)kv.first.second;
        hg.Nz = hg.P1; hg.M = hg.P2; hg.Ny = 1; hg.Nx = 2 * hg.P2;
        hg.n = (int64_t)hg.P1 * hg.P2;
        hg.rows = hg.P1;
        hg.w1c = 4;
        hg.w1r = row_w1(hg.M);
        hg.wx = row_w1(hg.M);
        const int P = hg.P1 * hg.P2;
        std::vector<double2> t64(P);
        std::vector<float2> t32(P);
        for (int m = 0; m < P; ++m) { t64[m] = root<double>(m, P); t32[m] = root<float>(m, P); }
        void* d64 = dalloc(p.get(), sizeof(double2) * P);
        void* d32 = dalloc(p.get(), sizeof(float2) * P);
        CK(cudaMemcpy(d64, t64.data(), sizeof(double2) * P, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d32, t32.data(), sizeof(float2) * P, cudaMemcpyHostToDevice));
        hg.twp64 = d64;
        hg.twp32 = d32;
        std::vector<int32_t> it(ids.begin(), ids.end());
        std::vector<int64_t> eo, so, co;
        for (int id : ids) { eo.push_back(p->eoff[id]); so.push_back(soff_c[id]); co.push_back(canon[id]); }
        int32_t* d_it = (int32_t*)dalloc(p.get(), sizeof(int32_t) * it.size());
        int64_t* d_eo = (int64_t*)dalloc(p.get(), sizeof(int64_t) * eo.size());
        int64_t* d_so = (int64_t*)dalloc(p.get(), sizeof(int64_t) * so.size());
        int64_t* d_co = (int64_t*)dalloc(p.get(), sizeof(int64_t) * co.size());
        CK(cudaMemcpy(d_it, it.data(), sizeof(int32_t) * it.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_eo, eo.data(), sizeof(int64_t) * eo.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_so, so.data(), sizeof(int64_t) * so.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_co, co.data(), sizeof(int64_t) * co.size(), cudaMemcpyHostToDevice));
        hg.g.ndim = 1; hg.g.Nz = hg.Nz; hg.g.Nmid = 1; hg.g.M = hg.M; hg.g.rows = hg.rows;
        hg.g.item = d_it; hg.g.eoff = d_eo; hg.g.soff = d_so; hg.g.coff = d_co;
        hg.d_canon = d_co;
        hg.h_soff = so;
        p->hgroups.push_back(hg);
      }
    }
    // Set the shared-memory attributes of every kernel the plan can launch
    // (both float32 tile widths).
    g_dry = true;
    try {
      Args a{};
      if (p->opts.pointwise) {
        g_pw_sel = true;
        for (const auto& dg : p->groups) {
          if (dg.ndim == 1) continue;   // the 1D passes read the bounds at run time
          launch_x<float>(XFWD, dg.M, dg.wx, a, dg.rows, 1, nullptr);
          launch_x<double>(XFWD, dg.M, dg.wx, a, dg.rows, 1, nullptr);
          launch_chk<float>(dg.Nz, dg.wc, a, dg.Ny, dg.M, 1, nullptr);
          launch_chk<double>(dg.Nz, dg.wc, a, dg.Ny, dg.M, 1, nullptr);
        }
        g_pw_sel = false;
      }
      if (p->opts.method != PV_POCS) {
        Args b{};
        b.pv = p->opts.method;
        for (const auto& dg : p->groups) {
          launch_x<float>(XPX, dg.M, dg.wx, b, dg.rows, 1, nullptr);
          launch_chk<float>(dg.Nz, dg.wc, b, dg.Ny, dg.M, 1, nullptr);
        }
      }
      for (const auto& dg0 : p->groups) {
        for (int alt = 0; alt < 3; ++alt) {
          DevGroup dg = dg0;
          dg.wa = dg.wc = alt == 2 ? -8 : alt ? 8 : 4;
          dg.w1c = alt ? 8 : 4;
          dg.wx = alt == 2 ? -row_w1(dg.M) : alt ? row_w2(dg.M) : row_w1(dg.M);
          dg.w1r = alt ? row_w2(dg.M) : row_w1(dg.M);
          if (ndim == 1) {
            launch_col1<float>(dg.P1, dg.w1c, a, dg.P2, 1, nullptr);
            launch_col1<double>(dg.P1, dg.w1c, a, dg.P2, 1, nullptr);
            launch_row1<float>(dg.P2, dg.w1r, a, dg.P1, 1, nullptr);
            launch_row1<double>(dg.P2, dg.w1r, a, dg.P1, 1, nullptr);
            continue;
          }
          launch_x<float>(XFWD, dg.M, dg.wx, a, dg.rows, 1, nullptr);
          launch_x<double>(XFWD, dg.M, dg.wx, a, dg.rows, 1, nullptr);
          launch_axis<float, -1>(dg.Ny < 8 ? 8 : dg.Ny, dg.wa, a, 1, dg.M, 1, nullptr);
          launch_axis<float, +1>(dg.Ny < 8 ? 8 : dg.Ny, dg.wa, a, 1, dg.M, 1, nullptr);
          launch_axis<double, -1>(dg.Ny < 8 ? 8 : dg.Ny, dg.wa, a, 1, dg.M, 1, nullptr);
          launch_axis<double, +1>(dg.Ny < 8 ? 8 : dg.Ny, dg.wa, a, 1, dg.M, 1, nullptr);
          launch_chk<float>(dg.Nz, dg.wc, a, dg.Ny, dg.M, 1, nullptr);
          launch_chk<double>(dg.Nz, dg.wc, a, dg.Ny, dg.M, 1, nullptr);
          launch_axis<float, +1>(dg.Nz, dg.wa, a, 1, dg.M, 1, nullptr);   // edit application
          launch_axis<float, -1>(dg.Nz, dg.wa, a, 1, dg.M, 1, nullptr);   // power-spectrum bounds
        }
      }
      for (const auto& hg : p->hgroups) {
        launch_col1<double>(hg.P1, hg.w1c, a, hg.P2, 1, nullptr);
        launch_row1<double>(hg.P2, hg.w1r, a, hg.P1, 1, nullptr);
      }
    } catch (...) {
      g_dry = false;
      g_pw_sel = false;
      throw;
    }
    g_dry = false;
    // float32 spectrum buffers: N/2 complex64 each (4 bytes per point)
    p->B32[0] = dalloc(p.get(), sizeof(float2) * p->total_c);
    p->B32[1] = dalloc(p.get(), sizeof(float2) * p->total_c);
    // projection variants: frequency residual (Dykstra, DR), q / u (Dykstra, ADMM)
    if (o.method == PV_DYKSTRA || o.method == PV_DR) p->pv_r = (float2*)dalloc(p.get(), sizeof(float2) * p->total_c);
    if (o.method == PV_DYKSTRA || o.method == PV_ADMM) {
      p->pv_q[0] = (float*)dalloc(p.get(), sizeof(float) * p->total);
      p->pv_q[1] = (float*)dalloc(p.get(), sizeof(float) * p->total);
    }
    build_tensor_maps(p.get());
    if (p->pv_r) build_aux_maps(p.get(), p->pv_r);
    p->d_prm = (ItemParams*)dalloc(p.get(), sizeof(ItemParams) * batch);
    p->d_st = (ItemState*)dalloc(p.get(), sizeof(ItemState) * batch);
    p->d_st2 = (ItemState*)dalloc(p.get(), sizeof(ItemState) * batch);
    p->d_nactive = (int*)dalloc(p.get(), sizeof(int));
    p->d_err = (int*)dalloc(p.get(), sizeof(int));
    {
      // per item: points, half-spectrum bins, and the offsets of the edit
      // arrays (1D items: bins of the layout of pointwise frequency bounds)
      p->ed_layout.resize(batch);
      std::array<int64_t, 6> acc{};
      for (int64_t i = 0; i < batch; ++i) {
        int64_t npt = 1, nb = 1;
        for (int d = 0; d < ndim; ++d) npt *= shapes[i * ndim + d];
        for (int d = 0; d < ndim - 1; ++d) nb *= shapes[i * ndim + d];
        nb *= shapes[i * ndim + ndim - 1] / 2 + 1;
        p->ed_layout[i] = {npt, nb, acc[2], acc[3], acc[4], acc[5]};
        acc[0] += npt; acc[1] += nb;
        acc[2] += (npt + 7) / 8; acc[3] += npt; acc[4] += (nb + 7) / 8; acc[5] += 2 * nb;
      }
      p->ed_total = acc;
    }
    if (p->opts.pointwise) {
      p->pw_e = (float*)dalloc(p.get(), sizeof(float) * p->total);
      p->pw_f = (float2*)dalloc(p.get(), sizeof(float2) * p->ed_total[1]);
      if (ndim > 1) {   // the check pass's packed layouts (1D passes read pw_f)
        p->pw_fp = (float2*)dalloc(p.get(), sizeof(float2) * p->total_c);
        build_aux_maps(p.get(), p->pw_fp);
        p->pw_f0 = (float4*)dalloc(p.get(), sizeof(float4) * p->total_rows);
      }
      p->pw_min = (unsigned int*)dalloc(p.get(), sizeof(unsigned int) * batch);
      p->pw_bad = (int*)dalloc(p.get(), sizeof(int));
    }
    if (p->opts.edits) {
      p->ed_s = (float*)dalloc(p.get(), sizeof(float) * p->total);
      p->ed_f = (float2*)dalloc(p.get(), sizeof(float2) * p->total_c);
      p->ed_p = (float2*)dalloc(p.get(), sizeof(float2) * p->total_c);
      p->ed_t = (int*)dalloc(p.get(), sizeof(int) * p->total_c);
      CK(cudaMemset(p->ed_s, 0, sizeof(float) * p->total));
      CK(cudaMemset(p->ed_f, 0, sizeof(float2) * p->total_c));
      CK(cudaMemset(p->ed_p, 0, sizeof(float2) * p->total_c));
      CK(cudaMemset(p->ed_t, 0, sizeof(int) * p->total_c));
    }
    CK(cudaMemset(p->d_err, 0, sizeof(int)));
    CK(cudaMallocHost(&p->h_err, sizeof(int)));
    p->d_loopcount = (int*)dalloc(p.get(), sizeof(int));
    CK(cudaMemset(p->d_st, 0, sizeof(ItemState) * batch));
    CK(cudaMemset(p->d_st2, 0, sizeof(ItemState) * batch));
    CK(cudaMallocHost(&p->h_nactive, sizeof(int)));
    CK(cudaMallocHost(&p->h_loopcount, sizeof(int)));
    CK(cudaMallocHost(&p->h_st, sizeof(ItemState) * batch));
    CK(cudaMallocHost(&p->h_prm, sizeof(ItemParams) * batch));
    {
      // placeholder bounds for the set-up launches below
      std::vector<double> one(batch, 1.0);
      upload_params(p.get(), one.data(), one.data(), 0, 0);
    }
    if (ndim == 1) {
      // chirp tables and FFT of the wrapped chirp of every item (float32 now,
      // float64 on first use)
      build_bt<float>(p.get());
      CK(cudaStreamSynchronize(p->stream));
    }
    build_multi(p.get());
    tune(p.get());   // tile widths only regroup pencils: Bt and the tables are unchanged
    *out = p.release();
    return FFCZ_OK;
  });
}

ffcz_status ffcz_set_stream(ffcz_plan_t plan, void* s) {
  if (!plan) return FFCZ_ERR_INVALID;
  plan->stream = (cudaStream_t)s;
  return FFCZ_OK;
}

size_t ffcz_workspace_bytes(ffcz_plan_t plan) { return plan ? plan->ws_bytes : 0; }

ffcz_status ffcz_edit_layout(ffcz_plan_t plan, int64_t item, int64_t* out) {
  if (!plan || !out) return FFCZ_ERR_INVALID;
  return guarded([&]() -> ffcz_status {
    if (item < -1 || item >= plan->batch) fail(FFCZ_ERR_INVALID, "item out of range");
    const auto& L = item < 0 ? plan->ed_total : plan->ed_layout[item];
    for (int k = 0; k < 6; ++k) out[k] = L[k];
    return FFCZ_OK;
  });
}

ffcz_status ffcz_edits_dense(ffcz_plan_t plan, float* s_dev, float* f_dev) {
  if (!plan) return FFCZ_ERR_INVALID;
  return guarded([&]() -> ffcz_status {
    if (!plan->opts.edits) fail(FFCZ_ERR_INVALID, "the plan was created without opts.edits");
    CK(cudaSetDevice(plan->device));
    if (s_dev)
      CK(cudaMemcpyAsync(s_dev, plan->ed_s, sizeof(float) * plan->total, cudaMemcpyDeviceToDevice, plan->stream));
    if (f_dev) {
      edits_canon(plan);
      CK(cudaMemcpyAsync(f_dev, plan->ed_canon, sizeof(float2) * plan->ed_total[1], cudaMemcpyDeviceToDevice,
                         plan->stream));
    }
    CK(cudaStreamSynchronize(plan->stream));
    CK(cudaGetLastError());
    return FFCZ_OK;
  });
}

ffcz_status ffcz_edits_compact(ffcz_plan_t plan, int m_bits, uint8_t* s_flags, int32_t* s_codes,
                               uint8_t* f_flags, int32_t* f_codes, int64_t* counts) {
  if (!plan) return FFCZ_ERR_INVALID;
  return guarded([&]() -> ffcz_status {
    if (!plan->opts.edits) fail(FFCZ_ERR_INVALID, "the plan was created without opts.edits");
    if (plan->opts.pointwise) fail(FFCZ_ERR_INVALID, "edit codes are relative to scalar bounds");
    if (m_bits < 2 || m_bits > 30) fail(FFCZ_ERR_INVALID, "m_bits must be in [2, 30]");
    if (!s_flags || !s_codes || !f_flags || !f_codes) fail(FFCZ_ERR_INVALID, "null edit array");
    CK(cudaSetDevice(plan->device));
    edits_compact(plan, m_bits, s_flags, s_codes, f_flags, f_codes, counts);
    return FFCZ_OK;
  });
}

ffcz_status ffcz_apply_edits(ffcz_plan_t plan, float* xhat_dev, const double* eps_s, const double* eps_f,
                             int m_bits, const uint8_t* s_flags, const int32_t* s_codes,
                             const uint8_t* f_flags, const int32_t* f_codes) {
  if (!plan) return FFCZ_ERR_INVALID;
  return guarded([&]() -> ffcz_status {
    if (plan->opts.pointwise) fail(FFCZ_ERR_INVALID, "edit codes are relative to scalar bounds");
    if (!xhat_dev || !eps_s || !eps_f || !s_flags || !s_codes || !f_flags || !f_codes)
      fail(FFCZ_ERR_INVALID, "null pointer argument");
    if (m_bits < 2 || m_bits > 30) fail(FFCZ_ERR_INVALID, "m_bits must be in [2, 30]");
    CK(cudaSetDevice(plan->device));
    upload_params(plan, eps_s, eps_f, 0, 0);
    apply_edits(plan, xhat_dev, m_bits, s_flags, s_codes, f_flags, f_codes);
    return FFCZ_OK;
  });
}

ffcz_status ffcz_edits_compact16(ffcz_plan_t plan, int m_bits, uint8_t* s_flags, int16_t* s_codes,
                                 int32_t* s_wide, uint8_t* f_flags, int16_t* f_codes, int32_t* f_wide,
                                 int64_t* counts) {
  if (!plan) return FFCZ_ERR_INVALID;
  return guarded([&]() -> ffcz_status {
    if (!plan->opts.edits) fail(FFCZ_ERR_INVALID, "the plan was created without opts.edits");
    if (plan->opts.pointwise) fail(FFCZ_ERR_INVALID, "edit codes are relative to scalar bounds");
    if (m_bits < 2 || m_bits > 16) fail(FFCZ_ERR_INVALID, "m_bits must be in [2, 16]");
    if (!s_flags || !s_codes || !s_wide || !f_flags || !f_codes || !f_wide) fail(FFCZ_ERR_INVALID, "null edit array");
    CK(cudaSetDevice(plan->device));
    edits_compact16(plan, m_bits, s_flags, s_codes, s_wide, f_flags, f_codes, f_wide, counts);
    return FFCZ_OK;
  });
}

ffcz_status ffcz_apply_edits16(ffcz_plan_t plan, float* xhat_dev, const double* eps_s, const double* eps_f,
                               int m_bits, const uint8_t* s_flags, const int16_t* s_codes, const int32_t* s_wide,
                               const uint8_t* f_flags, const int16_t* f_codes, const int32_t* f_wide,
                               const int64_t* counts) {
  if (!plan) return FFCZ_ERR_INVALID;
  return guarded([&]() -> ffcz_status {
    if (plan->opts.pointwise) fail(FFCZ_ERR_INVALID, "edit codes are relative to scalar bounds");
    if (!xhat_dev || !eps_s || !eps_f || !s_flags || !s_codes || !s_wide || !f_flags || !f_codes || !f_wide ||
        !counts)
      fail(FFCZ_ERR_INVALID, "null pointer argument");
    if (m_bits < 2 || m_bits > 16) fail(FFCZ_ERR_INVALID, "m_bits must be in [2, 16]");
    CK(cudaSetDevice(plan->device));
    upload_params(plan, eps_s, eps_f, 0, 0);
    apply_edits16(plan, xhat_dev, m_bits, s_flags, s_codes, s_wide, f_flags, f_codes, f_wide, counts);
    return FFCZ_OK;
  });
}

ffcz_status ffcz_power_spectrum_bounds(ffcz_plan_t plan, const float* x_dev, const double* rho, float* db_dev) {
  if (!plan) return FFCZ_ERR_INVALID;
  return guarded([&]() -> ffcz_status {
    if (!x_dev || !rho || !db_dev) fail(FFCZ_ERR_INVALID, "null pointer argument");
    for (int64_t i = 0; i < plan->batch; ++i)
      if (!(rho[i] > 0) || !std::isfinite(rho[i])) fail(FFCZ_ERR_INVALID, "rho must be finite and > 0");
    CK(cudaSetDevice(plan->device));
    ps_bounds(plan, x_dev, rho, reinterpret_cast<float2*>(db_dev));
    return FFCZ_OK;
  });
}

int ffcz_plan_describe(ffcz_plan_t plan, char* buf, int len) {
  if (!plan) return -1;
  std::string out;
  // a pass variant: tile width (tma(W): the persistent copy-engine-fed
  // kernel) and the radix split of its length, stage-1 x stage-2 sizes
  auto var = [](int w, int L) {
    const int S = (w > 0 && (w & kSplit)) ? 1 : 0;
    const int R1 = split_r1(L, S);
    const std::string split = " " + std::to_string(R1) + "x" + std::to_string(L / R1);
    if (w < 0) return "tma(" + std::to_string(-w) + ")" + split;
    return std::to_string(w & ~kSplit) + split;
  };
  for (const auto& dg : plan->groups) {
    char head[160];
    if (dg.ndim == 1)
      snprintf(head, sizeof head, "1d P=%dx%d count=%d:", dg.P1, dg.P2, dg.count);
    else if (dg.ndim == 2)
      snprintf(head, sizeof head, "2d %dx%d count=%d:", dg.Nz, dg.Nx, dg.count);
    else
      snprintf(head, sizeof head, "3d %dx%dx%d count=%d:", dg.Nz, dg.Ny, dg.Nx, dg.count);
    out += head;
    if (dg.ndim == 1) {
      out += " col1=" + var(dg.w1c, dg.P1) + " row1=" + var(dg.w1r, dg.P2);
    } else {
      out += " px=" + var(dg.wx, dg.M);
      if (dg.ndim == 3) out += " axis=" + var(dg.wa, dg.Ny);
      out += " chk=" + var(dg.wc, dg.Nz);
    }
    out += "\n";
  }
  {
    std::string mk;
    for (int k = 0; k < MK_N; ++k)
      if (plan->mp[k].n) mk += std::string(" ") + multi_name(k) + "=" + (plan->multi_use[k] ? "multi" : "separate");
    if (!mk.empty()) out += "passes over all groups:" + mk + "\n";
  }
  if (buf && len > 0) {
    const size_t n = std::min(out.size(), (size_t)len - 1);
    memcpy(buf, out.data(), n);
    buf[n] = 0;
  }
  return (int)out.size();
}

ffcz_status ffcz_correct(ffcz_plan_t plan, float* e, const double* eps_s, const double* eps_f,
                         ffcz_stats* stats) {
  if (!plan) return FFCZ_ERR_INVALID;
  return guarded([&]() {
    if (plan->opts.pointwise) fail(FFCZ_ERR_INVALID, "pointwise plan: use ffcz_correct_pw");
    return correct_impl(plan, e, eps_s, eps_f, stats);
  });
}

ffcz_status ffcz_correct_pw(ffcz_plan_t plan, float* e, const float* eb, const float* db, ffcz_stats* stats) {
  if (!plan) return FFCZ_ERR_INVALID;
  return guarded([&]() {
    if (!plan->opts.pointwise) fail(FFCZ_ERR_INVALID, "the plan was created without opts.pointwise");
    if (!e || !eb || !db) fail(FFCZ_ERR_INVALID, "null pointer argument");
    CK(cudaSetDevice(plan->device));
    CK(cudaMemcpyAsync(plan->pw_e, eb, sizeof(float) * plan->total, cudaMemcpyDeviceToDevice, plan->stream));
    CK(cudaMemcpyAsync(plan->pw_f, db, sizeof(float2) * plan->ed_total[1], cudaMemcpyDeviceToDevice,
                       plan->stream));
    std::vector<double> ones(plan->batch, 1.0);   // the item bounds become ratios
    return correct_impl(plan, e, ones.data(), ones.data(), stats);
  });
}

ffcz_status ffcz_correct_host(ffcz_plan_t plan, float* e_host, const double* eps_s,
                              const double* eps_f, ffcz_stats* stats) {
  if (!plan) return FFCZ_ERR_INVALID;
  return guarded([&]() -> ffcz_status {
    if (plan->opts.pointwise) fail(FFCZ_ERR_INVALID, "pointwise plan: use ffcz_correct_pw");
    if (!e_host) fail(FFCZ_ERR_INVALID, "e_host is null");
    CK(cudaSetDevice(plan->device));
    if (!plan->staging) plan->staging = (float*)dalloc(plan, sizeof(float) * plan->total);
    if (spec_upload(plan, plan->staging, e_host))
      return correct_impl(plan, plan->staging, eps_s, eps_f, stats, e_host, true);
    CK(cudaMemcpyAsync(plan->staging, e_host, sizeof(float) * plan->total, cudaMemcpyHostToDevice,
                       plan->stream));
    return correct_impl(plan, plan->staging, eps_s, eps_f, stats, e_host);
  });
}

ffcz_status ffcz_check(ffcz_plan_t plan, const float* e, const double* eps_s, const double* eps_f,
                       ffcz_stats* stats) {
  if (!plan) return FFCZ_ERR_INVALID;
  return guarded([&]() -> ffcz_status {
    if (plan->opts.pointwise) fail(FFCZ_ERR_INVALID, "pointwise plan: use ffcz_correct_pw");
    if (!e || !eps_s || !eps_f) fail(FFCZ_ERR_INVALID, "null pointer argument");
    CK(cudaSetDevice(plan->device));
    ProfOn prof_on(plan);
    upload_params(plan, eps_s, eps_f, 0, 0);
    CK(cudaEventRecord(plan->ev0, plan->stream));
    cert_reset(plan);
    certify(plan, e, false);
    CK(cudaEventRecord(plan->ev2, plan->stream));
    CK(cudaEventSynchronize(plan->ev2));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, plan->ev0, plan->ev2));
    fill_stats(plan, stats, ms, ms, true);
    if (stats)
      for (int64_t i = 0; i < plan->batch; ++i) { stats[i].iters = 0; stats[i].status = 0; }
    CK(cudaGetLastError());
    for (int64_t i = 0; i < plan->batch; ++i)
      if (!plan->h_st[i].certified) return FFCZ_ERR_CERT_FAILED;
    return FFCZ_OK;
  });
}

ffcz_status ffcz_correct_backward(ffcz_plan_t plan, const float* e0, const float* gout, float* gin,
                                  const double* eps_s, const double* eps_f) {
  if (!plan) return FFCZ_ERR_INVALID;
  return guarded([&]() { return backward_impl(plan, e0, gout, gin, eps_s, eps_f); });
}

int64_t ffcz_ckpt_floats(ffcz_plan_t plan) {
  if (!plan || plan->opts.K < 1 || plan->opts.ckpt_every < 1) return 0;
  return (int64_t)((plan->opts.K + plan->opts.ckpt_every - 1) / plan->opts.ckpt_every) * plan->total;
}

ffcz_status ffcz_correct_ckpt(ffcz_plan_t plan, float* e, const double* eps_s, const double* eps_f,
                              float* ckpt, ffcz_stats* stats) {
  if (!plan) return FFCZ_ERR_INVALID;
  return guarded([&]() -> ffcz_status {
    bw_check(plan);
    if (!e || !ckpt) fail(FFCZ_ERR_INVALID, "null pointer argument");
    const ffcz_opts& o = plan->opts;
    if (o.min_iters != o.K || o.max_iters != o.K || o.precision != 32 || o.certify)
      fail(FFCZ_ERR_INVALID, "the differentiable forward needs min_iters = max_iters = K, precision 32 "
                             "and no certification");
    CK(cudaSetDevice(plan->device));
    bw_alloc(plan);
    plan->km_valid = false;
    if (o.keep_masks && plan->km_K != o.K) {
      // one mask block per step t = 0..K (x-pass masks of steps 1..K,
      // check-pass masks of checks 0..K - 1)
      plan->km_s = (uint32_t*)dalloc(plan, sizeof(uint32_t) * plan->px_words * (o.K + 1));
      plan->km_f = (uint32_t*)dalloc(plan, sizeof(uint32_t) * plan->chk_words * (o.K + 1));
      plan->km_K = o.K;
    }
    plan->ck_rec = true;
    struct Off { ffcz_plan_s* p; ~Off() { p->ck_rec = false; } } off{plan};
    const ffcz_status st = correct_impl(plan, e, eps_s, eps_f, stats);
    CK(cudaMemcpyAsync(ckpt, plan->bw_ck, sizeof(float) * ffcz_ckpt_floats(plan), cudaMemcpyDeviceToDevice,
                       plan->stream));
    CK(cudaStreamSynchronize(plan->stream));
    plan->km_valid = o.keep_masks && plan->km_K == o.K;
    return st;
  });
}

ffcz_status ffcz_correct_backward_ckpt(ffcz_plan_t plan, const float* e0, const float* ckpt, const float* gout,
                                       float* gin, const double* eps_s, const double* eps_f) {
  if (!plan) return FFCZ_ERR_INVALID;
  return guarded([&]() {
    if (!ckpt) fail(FFCZ_ERR_INVALID, "null pointer argument");
    return backward_impl(plan, e0, gout, gin, eps_s, eps_f, ckpt);
  });
}

void ffcz_destroy(ffcz_plan_t plan) {
  if (plan) free_plan(plan);
}

const char* ffcz_strerror(ffcz_status s) {
  switch (s) {
    case FFCZ_OK: return "ok";
    case FFCZ_ERR_INVALID: return "invalid argument";
    case FFCZ_ERR_UNSUPPORTED: return "unsupported shape or option";
    case FFCZ_ERR_CUDA: return "CUDA error";
    case FFCZ_ERR_NOT_CONVERGED: return "not converged within max_iters";
    case FFCZ_ERR_CERT_FAILED: return "FP64 certification failed";
    case FFCZ_ERR_NONFINITE: return "non-finite value in the error field or its spectrum";
    case FFCZ_ERR_TIMEOUT: return "bounded device wait timed out";
    case FFCZ_ERR_OOM: return "out of device memory";
  }
  return "unknown status";
}

const char* ffcz_last_error(void) { return g_err.c_str(); }

ffcz_status ffcz_profile_enable(ffcz_plan_t plan, int on) {
  if (!plan) return FFCZ_ERR_INVALID;
  plan->prof = on != 0;
  plan->prof_tab.clear();
  plan->prof_keys.clear();
  return FFCZ_OK;
}

int ffcz_profile_count(ffcz_plan_t plan) { return plan ? (int)plan->prof_keys.size() : 0; }

ffcz_status ffcz_profile_entry(ffcz_plan_t plan, int i, char* name, int name_len, double* ms,
                               int64_t* launches) {
  if (!plan || i < 0 || i >= (int)plan->prof_keys.size() || !name || name_len < 1)
    return FFCZ_ERR_INVALID;
  const std::string& k = plan->prof_keys[i];
  snprintf(name, (size_t)name_len, "%s", k.c_str());
  const auto& v = plan->prof_tab[k];
  if (ms) *ms = v.first;
  if (launches) *launches = v.second;
  return FFCZ_OK;
}

int64_t ffcz_launch_count(void) { return g_launches.load(); }

ffcz_status ffcz_fp64_peak(int kind, void* cuda_stream, double* flops_per_s) {
  return guarded([&]() -> ffcz_status {
    if (!flops_per_s || (kind != 0 && kind != 1)) fail(FFCZ_ERR_INVALID, "kind must be 0 or 1, flops_per_s non-null");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    double* out = nullptr;
    CK(cudaMalloc(&out, sizeof(double)));
    cudaEvent_t a = nullptr, b = nullptr;
    const int blocks = sms * 8, threads = 256, iters = 4096;
    float best = 0.f;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(a, s);
      k_fp64_peak<<<blocks, threads, 0, s>>>(out, iters, kind, 1.0000000001, 1e-9);
      g_launches++;
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(b, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;   // rep 0 warms up
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) fail(FFCZ_ERR_CUDA, cudaGetErrorString(e));
    const double ops = (double)blocks * threads * kFpChains * iters;
    *flops_per_s = ops * (kind == 0 ? 2.0 : 1.0) / (best * 1e-3);
    return FFCZ_OK;
  });
}

}  // extern "C"
