// noalloc.cu -- ffcz_check_static: the FP64 certification check for one
// field, with no plan and no device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// check: hosts whose memory manager (a framework's caching allocator, a
// memory pool sized at start-up) owns the whole device so that no other
// allocation may happen, callback-driven pipelines that must not reach the
// allocator, and validation steps that must not fail for lack of memory in
// the middle of a run.  For them this entry point keeps its scratch (twiddle
// tables, loop state, the float64 spectrum) in one file-scope __device__
// array of fixed size.  Every device that loads the library holds that array
// until the process exits.
//
// Contract (also in include/ffcz.h):
//  * The first call on each device sets that device up: it takes the array's
//    device address with cudaGetSymbolAddress, copies the twiddle tables into
//    it and makes the runtime load every kernel this entry point launches
//    (so that no later call loads code).  Make that first call before any
//    stream capture begins.
//  * Each call waits for its stream before returning (the stats are read
//    back to the host).
//  * Every call on a device shares the same array; calls whose GPU work
//    overlaps (other streams, other host threads) race and may return wrong
//    results.  Calls ordered on one stream are safe.
//  * Fields larger than FFCZ_STATIC_MAX_POINTS points are rejected with
//    FFCZ_ERR_INVALID before any GPU work.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ffcz.h"
#include "passes.cuh"

using namespace ffcz;

__attribute__((visibility("hidden"))) void ffcz_set_last_error(const char* msg);

namespace {

// Scratch layout: [tables][group arrays][params][state][float64 spectrum].
constexpr size_t kTablesBytes = 256 * 1024;
constexpr size_t kHeadBytes = 4096;   // group arrays + params + state
constexpr size_t kSpecBytes = (size_t)FFCZ_STATIC_MAX_POINTS * 8;   // n/2 complex doubles
constexpr size_t kScratchBytes = kTablesBytes + kHeadBytes + kSpecBytes;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// Detail message for ffcz_last_error() (defined in ffcz.cu).
struct ErrSink {
  std::string msg;
  ErrSink& operator=(const std::string& m) { msg = m; ffcz_set_last_error(msg.c_str()); return *this; }
  ErrSink& operator=(const char* m) { return *this = std::string(m); }
  void clear() { msg.clear(); ffcz_set_last_error(""); }
};
thread_local ErrSink s_err;

struct DevSetup {
  bool ready = false;
  unsigned char* base = nullptr;            // device address of g_static_scratch
  const void* stage_tab[12] = {};           // float64 stage-2 twiddles, L = 2^p
  const void* r2c_tab[12] = {};             // float64 R2C factors, Nx = 2^p
};
constexpr int kMaxDev = 64;
DevSetup s_dev[kMaxDev];
std::mutex s_mu;

long double twopi() { return 2.0L * acosl(-1.0L); }

void root_ld(long double m, long double L, long double& c, long double& s) {
  const long double a = twopi() * m / L;
  c = cosl(a);
  s = -sinl(a);
  if (fabsl(c) < 1e-18L) c = 0.0L;
  if (fabsl(s) < 1e-18L) s = 0.0L;
}

double2 root64(long double m, long double L) {
  long double c, s;
  root_ld(m, L, c, s);
  return make_double2((double)c, (double)s);
}

// Stage-2 twiddles of the two-stage split of L (layout in fft_core.cuh; the
// factors t >= R2/2 in tangent form).
void stage_factors_rt(int L, std::vector<double2>& out) {
  const int R1 = f2_nt(L), R2 = L / R1;
  out.assign(L, make_double2(0.0, 0.0));
  for (int k1 = 0; k1 < R1; ++k1)
    for (int t = 1; t < R2; ++t) {
      long double c, s;
      root_ld((long double)k1 * t, (long double)L, c, s);
      out[tw_index(R1, k1, t)] = f64_stage_entry(c, s, t >= R2 / 2);
    }
}

// Queries the kernel's attributes, which makes a lazily loading runtime load
// it now rather than at its first launch, and raises its dynamic shared
// memory limit where it needs more than the default 48 KiB.
template <typename K>
cudaError_t allow_smem(K k, size_t bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k);
  if (e != cudaSuccess || bytes <= 48 * 1024) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int L>
cudaError_t allow_all() {
  cudaError_t e = allow_smem(k_xfwd<double, L>, Smem<double, L>::bytes_x);
  if (e == cudaSuccess) e = allow_smem(k_axis<double, L, -1>, Smem<double, L>::bytes_axis);
  if (e == cudaSuccess) e = allow_smem(k_chk<double, L>, Smem<double, L>::bytes_axis);
  return e;
}

__global__ void k_static_init(int32_t* item, int64_t* eoff, int64_t* soff, ItemParams* prm,
                              ItemState* st, ItemParams p);

// Once per device, with that device current.
bool setup(int dev, DevSetup*& out) {
  if (dev < 0 || dev >= kMaxDev) { s_err = "device ordinal out of range"; return false; }
  std::lock_guard<std::mutex> lk(s_mu);
  DevSetup& d = s_dev[dev];
  if (d.ready) { out = &d; return true; }
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
  if (e != cudaSuccess) {
    s_err = std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e);
    return false;
  }
  d.base = static_cast<unsigned char*>(ptr);
  size_t off = 0;
  std::vector<double2> tab;
  for (int p = 3; p <= 10; ++p) {
    stage_factors_rt(1 << p, tab);
    const size_t bytes = tab.size() * sizeof(double2);
    e = cudaMemcpy(d.base + off, tab.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { s_err = std::string("table upload: ") + cudaGetErrorString(e); return false; }
    d.stage_tab[p] = d.base + off;
    off += (bytes + 255) & ~size_t(255);
  }
  for (int p = 4; p <= 11; ++p) {
    const int Nx = 1 << p;
    tab.assign(Nx / 2, make_double2(0.0, 0.0));
    for (int k = 0; k < Nx / 2; ++k) tab[k] = root64(k, Nx);
    const size_t bytes = tab.size() * sizeof(double2);
    e = cudaMemcpy(d.base + off, tab.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { s_err = std::string("table upload: ") + cudaGetErrorString(e); return false; }
    d.r2c_tab[p] = d.base + off;
    off += (bytes + 255) & ~size_t(255);
  }
  if (off > kTablesBytes) { s_err = "static table area too small"; return false; }
  e = allow_all<8>();
  if (e == cudaSuccess) e = allow_all<16>();
  if (e == cudaSuccess) e = allow_all<32>();
  if (e == cudaSuccess) e = allow_all<64>();
  if (e == cudaSuccess) e = allow_all<128>();
  if (e == cudaSuccess) e = allow_all<256>();
  if (e == cudaSuccess) e = allow_all<512>();
  if (e == cudaSuccess) e = allow_all<1024>();
  if (e == cudaSuccess) e = allow_smem(k_static_init, 0);
  if (e == cudaSuccess) e = allow_smem(k_certify, 0);
  if (e != cudaSuccess) { s_err = std::string("kernel attributes: ") + cudaGetErrorString(e); return false; }
  d.ready = true;
  out = &d;
  return true;
}

// Writes the per-call header (group arrays, parameters, cleared state).
__global__ void k_static_init(int32_t* item, int64_t* eoff, int64_t* soff, ItemParams* prm,
                              ItemState* st, ItemParams p) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  item[0] = 0;
  eoff[0] = 0;
  soff[0] = 0;
  prm[0] = p;
  ItemState z;
  memset(&z, 0, sizeof(z));
  st[0] = z;
}

template <int M>
void launch_xfwd(const Args& a, int64_t rows, cudaStream_t s) {
  using G_ = Geo<double, M>;
  dim3 grid((unsigned)(((rows + G_::W - 1) / G_::W + G_::G - 1) / G_::G), 1);
  k_xfwd<double, M><<<grid, G_::NTHR, Smem<double, M>::bytes_x, s>>>(a);
}
template <int L>
void launch_axis(const Args& a, int Nz, int M, cudaStream_t s) {
  using G_ = Geo<double, L>;
  dim3 grid((unsigned)(((int64_t)Nz * (M / G_::W) + G_::G - 1) / G_::G), 1);
  k_axis<double, L, -1><<<grid, G_::NTHR, Smem<double, L>::bytes_axis, s>>>(a);
}
template <int L>
void launch_chk(const Args& a, int Nmid, int M, cudaStream_t s) {
  using G_ = Geo<double, L>;
  dim3 grid((unsigned)((chk_ntiles(G_::W, M, Nmid) + G_::G - 1) / G_::G), 1);
  k_chk<double, L><<<grid, G_::NTHR, Smem<double, L>::bytes_axis, s>>>(a);
}

#define FFCZ_SWITCH_L(n, CALL)              \
  switch (n) {                              \
    case 8: CALL(8); break;                 \
    case 16: CALL(16); break;               \
    case 32: CALL(32); break;               \
    case 64: CALL(64); break;               \
    case 128: CALL(128); break;             \
    case 256: CALL(256); break;             \
    case 512: CALL(512); break;             \
    case 1024: CALL(1024); break;           \
    default: break;                         \
  }

bool pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

ffcz_status run(const float* e, int ndim, const int64_t* shape, double E, double D, void* stream,
                ffcz_stats* out) {
  if (!e || !shape) { s_err = "null pointer argument"; return FFCZ_ERR_INVALID; }
  if (ndim != 2 && ndim != 3) { s_err = "ndim must be 2 or 3"; return FFCZ_ERR_INVALID; }
  int64_t n = 1;
  for (int d = 0; d < ndim; ++d) {
    const int64_t v = shape[d];
    const bool last = d == ndim - 1;
    if (!pow2(v) || v < (last ? 16 : 8) || v > (last ? 2048 : 1024)) {
      s_err = "axis lengths must be powers of two in [8, 1024] ([16, 2048] for the last axis)";
      return FFCZ_ERR_UNSUPPORTED;
    }
    n *= v;
  }
  if (n > (int64_t)FFCZ_STATIC_MAX_POINTS) {
    s_err = "field of " + std::to_string(n) + " points exceeds the static scratch limit of " +
            std::to_string((long long)FFCZ_STATIC_MAX_POINTS) + " points";
    return FFCZ_ERR_INVALID;
  }
  if (!(E > 0) || !(D > 0) || !std::isfinite(E) || !std::isfinite(D)) {
    s_err = "bounds must be finite and > 0";
    return FFCZ_ERR_INVALID;
  }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) { s_err = std::string(cudaGetErrorString(ce)); return FFCZ_ERR_CUDA; }
  DevSetup* ds = nullptr;
  if (!setup(dev, ds)) return FFCZ_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;

  unsigned char* head = ds->base + kTablesBytes;
  int32_t* item = reinterpret_cast<int32_t*>(head);
  int64_t* eoff = reinterpret_cast<int64_t*>(head + 256);
  int64_t* soff = reinterpret_cast<int64_t*>(head + 512);
  ItemParams* prm = reinterpret_cast<ItemParams*>(head + 1024);
  ItemState* st = reinterpret_cast<ItemState*>(head + 2048);
  void* spec = ds->base + kTablesBytes + kHeadBytes;

  const int Nx = (int)shape[ndim - 1], M = Nx / 2, Nz = (int)shape[0];
  const int Ny = ndim == 3 ? (int)shape[1] : 1;
  ItemParams q{};
  q.E = E; q.D = D; q.Es = E; q.Ds = D; q.thr = D; q.inv_n = 1.0 / (double)n;
  q.Esf = (float)E; q.Dsf = (float)D; q.thrf = (float)D; q.inv_nf = (float)q.inv_n;
  q.n = n; q.min_iters = 0; q.max_iters = 0; q.bscale = 1.0;
  k_static_init<<<1, 32, 0, s>>>(item, eoff, soff, prm, st, q);

  Args a{};
  a.g.ndim = ndim; a.g.Nz = Nz; a.g.Nmid = Ny; a.g.M = M; a.g.rows = n / Nx;
  a.g.item = item; a.g.eoff = eoff; a.g.soff = soff;
  a.prm = prm; a.st = st; a.B0 = spec; a.B1 = spec;
  a.e = const_cast<float*>(e);
  a.pred = P_ALL; a.sel_in = a.sel_out = S_CUR;
  a.mode = M_MEASURE;
  a.tw = ds->stage_tab[ilog2(M)];
  a.twr = ds->r2c_tab[ilog2(Nx)];
  const int64_t rows = n / Nx;
#define X_(K) launch_xfwd<K>(a, rows, s)
  FFCZ_SWITCH_L(M, X_)
#undef X_
  a.mode = 0;
  if (ndim == 3) {
    a.tw = ds->stage_tab[ilog2(Ny)];
#define A_(K) launch_axis<K>(a, Nz, M, s)
    FFCZ_SWITCH_L(Ny, A_)
#undef A_
  }
  a.tw = ds->stage_tab[ilog2(Nz)];
  a.mode = M_NOWRITE;
#define C_(K) launch_chk<K>(a, Ny, M, s)
  FFCZ_SWITCH_L(Nz, C_)
#undef C_
  k_certify<<<1, 32, 0, s>>>(prm, st, 1, 0);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) { s_err = std::string("launch: ") + cudaGetErrorString(ce); return FFCZ_ERR_CUDA; }
  ItemState h;
  ce = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) { s_err = std::string("readback: ") + cudaGetErrorString(ce); return FFCZ_ERR_CUDA; }
  if (out) {
    memset(out, 0, sizeof(*out));
    out->certified = h.certified;
    out->s_ratio = h.emax64 / E;
    out->f_margin64 = 1.0 - (h.v64 + h.bound64) / D;
    out->s_margin64 = 1.0 - h.emax64 / E;
  }
  return h.certified ? FFCZ_OK : FFCZ_ERR_CERT_FAILED;
}

}  // namespace

extern "C" ffcz_status ffcz_check_static(const float* e_dev, int ndim, const int64_t* shape,
                                         double eps_s, double eps_f, void* cuda_stream,
                                         ffcz_stats* stats) {
  s_err.clear();
  try {
    return run(e_dev, ndim, shape, eps_s, eps_f, cuda_stream, stats);
  } catch (...) {
    s_err = "unexpected host exception";
    return FFCZ_ERR_CUDA;
  }
}
