// edits.cuh -- storage form of the Alg. 1 edits (Sec. IV-B, "Compaction,
// quantization, and lossless compression of edits"; the lossless back end
// is not part of this library).
//
// Canonical layout: spatial edits like the field (float32 per point);
// frequency edits as the half spectrum of a real-input FFT, complex64
// [Nz][Ny][Nx/2+1] per item (2D: [Ny][Nx/2+1]).
// CompactEdits: flags = 1 where a component is nonzero (a complex bin counts
// once), packed 8 per byte, first component in bit 0; compact edits = the
// nonzero components in order.  QuantizeEdits: code = rint(edit / q),
// q = 2 bound / 2^m, division and rounding in float32, Re and Im coded
// separately.  Items are compacted independently into fixed regions.
#pragma once
#include "passes.cuh"

namespace ffcz {

// Packed spectrum (kx = 0 slot = A + iB, A, B the kx = 0 and kx = Nx/2
// planes) -> canonical half spectrum.  Grid (x: bins, y: group members).
static __global__ void k_edits_canon(Group g, const float2* ed_f, float2* out, const int64_t* ooff) {
  const int gi = blockIdx.y;
  const int Nz = g.Nz, Ny = g.Nmid, M = g.M;
  const int64_t nb = (int64_t)Nz * Ny * (M + 1);
  const float2* F = ed_f + g.soff[gi];
  float2* o = out + ooff[gi];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % (M + 1));
    const int64_t r = i / (M + 1);               // kz Ny + ky
    if (kx > 0 && kx < M) {
      o[i] = F[r * M + kx];
      continue;
    }
    const int ky = (int)(r % Ny), kz = (int)(r / Ny);
    const int64_t rm = (int64_t)((Nz - kz) % Nz) * Ny + (Ny - ky) % Ny;
    const float2 c = F[r * M], cm = F[rm * M];
    // A = (C + conj Cm) / 2, B = (C - conj Cm) / (2i)
    o[i] = kx == 0 ? make_float2(0.5f * (c.x + cm.x), 0.5f * (c.y - cm.y))
                   : make_float2(0.5f * (c.y + cm.y), -0.5f * (c.x - cm.x));
  }
}

__device__ __forceinline__ bool nz_comp(float v) { return v != 0.f; }
__device__ __forceinline__ bool nz_comp(float2 v) { return v.x != 0.f || v.y != 0.f; }

// One region to compact: n components at `vals`, flags at `flags`, codes at
// `codes`, chunk counts at `chunks`, step q.
template <typename C>
struct EdRegion {
  const C* vals;
  int64_t n;
  uint8_t* flags;
  int32_t* codes;
  int* chunks;
  float q;
};

constexpr int kEdThreads = 256;
constexpr int kEdChunk = kEdThreads * 8;   // components per CTA

// Flags and per-chunk counts.  Each thread owns 8 consecutive components
// (one flag byte).
template <typename C>
static __global__ void k_edits_count(const EdRegion<C>* regs) {
  const EdRegion<C> r = regs[blockIdx.y];
  const int64_t c0 = (int64_t)blockIdx.x * kEdChunk;
  if (c0 >= r.n) return;
  const int64_t b = c0 / 8 + threadIdx.x;     // flag byte
  int cnt = 0;
  if (b * 8 < r.n) {
    unsigned byte = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t i = b * 8 + k;
      if (i < r.n && nz_comp(r.vals[i])) byte |= 1u << k;
    }
    r.flags[b] = (uint8_t)byte;
    cnt = __popc(byte);
  }
  __shared__ int s[kEdThreads / 32];
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kEdThreads / 32; ++w) t += s[w];
    r.chunks[blockIdx.x] = t;
  }
}

// Exclusive scan of the chunk counts of each region (one CTA per region);
// the region's total goes to totals[region].
template <typename C>
static __global__ void k_edits_scan(const EdRegion<C>* regs, int64_t* totals) {
  const EdRegion<C> r = regs[blockIdx.x];
  const int64_t nch = (r.n + kEdChunk - 1) / kEdChunk;
  __shared__ long long carry;
  __shared__ long long s[1024];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nch; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const long long v = i < nch ? r.chunks[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {   // inclusive Hillis-Steele scan
      const long long add = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < nch) r.chunks[i] = (int)(carry + s[threadIdx.x] - v);
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += s[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

__device__ __forceinline__ int32_t quant_code(float v, float q) {
  const float r = rintf(v / q);                // IEEE division, ties to even
  return (int32_t)fminf(fmaxf(r, -2147483520.f), 2147483520.f);
}
__device__ __forceinline__ void put_codes(int32_t* codes, int64_t k, float v, float q) { codes[k] = quant_code(v, q); }
__device__ __forceinline__ void put_codes(int32_t* codes, int64_t k, float2 v, float q) {
  codes[2 * k] = quant_code(v.x, q);
  codes[2 * k + 1] = quant_code(v.y, q);
}

// Quantized nonzero components at their compacted positions.
template <typename C>
static __global__ void k_edits_scatter(const EdRegion<C>* regs) {
  const EdRegion<C> r = regs[blockIdx.y];
  const int64_t c0 = (int64_t)blockIdx.x * kEdChunk;
  if (c0 >= r.n) return;
  const int64_t b = c0 / 8 + threadIdx.x;
  const unsigned byte = (b * 8 < r.n) ? r.flags[b] : 0u;
  const int cnt = __popc(byte);
  // block exclusive scan of the per-thread counts
  __shared__ int s[kEdThreads / 32];
  int incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if ((threadIdx.x & 31) >= (unsigned)o) incl += y;
  }
  if ((threadIdx.x & 31) == 31) s[threadIdx.x >> 5] = incl;
  __syncthreads();
  int wbase = 0;
  for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wbase += s[w];
  int64_t k = (int64_t)r.chunks[blockIdx.x] + wbase + incl - cnt;
#pragma unroll
  for (int t = 0; t < 8; ++t)
    if (byte & (1u << t)) put_codes(r.codes, k++, r.vals[b * 8 + t], r.q);
}

// ----- 16-bit storage of the codes (m <= 16) -----------------------------------
// A code in [-32767, 32767] is stored as itself in int16; any other code (the
// end point 2^15 of m = 16, or an edit beyond the bound) as the escape -32768,
// with its value appended, in order of appearance, to an int32 list.

constexpr int16_t kEscape16 = -32768;
__device__ __forceinline__ bool code_escapes(int32_t c) { return c < -32767 || c > 32767; }

// One region of codes: narrowing reads c32 and writes c16 + wide; widening
// reads c16 + wide (nwide entries) and writes c32.
struct CodeRegion {
  int32_t* c32;
  int16_t* c16;
  int32_t* wide;
  int64_t n;       // codes in the region
  int64_t nwide;   // widening: entries of the list
  int* chunks;     // escapes per chunk of kEdChunk codes -> exclusive offsets
};

// Block-wide exclusive scan of nch chunk counts in place (blockDim.x = 1024);
// returns the total to every thread.
__device__ long long scan_chunks(int* chunks, int64_t nch) {
  __shared__ long long carry;
  __shared__ long long s[1024];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nch; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const long long v = i < nch ? chunks[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {   // inclusive Hillis-Steele scan
      const long long add = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < nch) chunks[i] = (int)(carry + s[threadIdx.x] - v);
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += s[threadIdx.x];
    __syncthreads();
  }
  return carry;
}

// Escapes per chunk; each thread owns 8 consecutive codes.
template <bool NARROW>
static __global__ void k_codes_count(const CodeRegion* regs) {
  const CodeRegion r = regs[blockIdx.y];
  const int64_t c0 = (int64_t)blockIdx.x * kEdChunk;
  if (c0 >= r.n) return;
  const int64_t i0 = c0 + (int64_t)threadIdx.x * 8;
  int cnt = 0;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int64_t i = i0 + t;
    if (i < r.n) cnt += NARROW ? (int)code_escapes(r.c32[i]) : (int)(r.c16[i] == kEscape16);
  }
  __shared__ int s[kEdThreads / 32];
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kEdThreads / 32; ++w) t += s[w];
    r.chunks[blockIdx.x] = t;
  }
}

// Exclusive offsets of the chunks of each region (one CTA per region); the
// region's escape count goes to totals[region].
static __global__ void k_codes_scan(const CodeRegion* regs, int64_t* totals) {
  const CodeRegion r = regs[blockIdx.x];
  const long long t = scan_chunks(r.chunks, (r.n + kEdChunk - 1) / kEdChunk);
  if (threadIdx.x == 0) totals[blockIdx.x] = t;
}

// Narrowing: int16 codes and the escaped values at their list positions.
// Widening: int32 codes, an escape taking the list entry of its rank (the
// host has checked that the escapes number exactly nwide).
template <bool NARROW>
static __global__ void k_codes_scatter(const CodeRegion* regs) {
  const CodeRegion r = regs[blockIdx.y];
  const int64_t c0 = (int64_t)blockIdx.x * kEdChunk;
  if (c0 >= r.n) return;
  const int64_t i0 = c0 + (int64_t)threadIdx.x * 8;
  unsigned esc = 0;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int64_t i = i0 + t;
    if (i < r.n && (NARROW ? code_escapes(r.c32[i]) : r.c16[i] == kEscape16)) esc |= 1u << t;
  }
  const int cnt = __popc(esc);
  __shared__ int s[kEdThreads / 32];
  int incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if ((threadIdx.x & 31) >= (unsigned)o) incl += y;
  }
  if ((threadIdx.x & 31) == 31) s[threadIdx.x >> 5] = incl;
  __syncthreads();
  int wbase = 0;
  for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wbase += s[w];
  int64_t k = (int64_t)r.chunks[blockIdx.x] + wbase + incl - cnt;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int64_t i = i0 + t;
    if (i >= r.n) break;
    const bool e = (esc >> t) & 1u;
    if constexpr (NARROW) {
      const int32_t c = r.c32[i];
      r.c16[i] = e ? kEscape16 : (int16_t)c;
      if (e) r.wide[k] = c;
    } else {
      r.c32[i] = e ? (k < r.nwide ? r.wide[k] : 0) : (int32_t)r.c16[i];
    }
    k += e;
  }
}

// ----- power-spectrum relative bounds (reading: the per-shell positive root) -------
// Shell of a canonical bin (kz, ky, kx): rounded radius of the signed
// frequency vector; kx in [0, M] is already non-negative.
__device__ __forceinline__ int ps_shell(int kz, int ky, int kx, int Nz, int Ny) {
  const int sz = kz <= Nz / 2 ? kz : kz - Nz, sy = ky <= Ny / 2 ? ky : ky - Ny;
  return (int)rint(sqrt((double)kx * kx + (double)sy * sy + (double)sz * sz));
}

// Per-item shell sums over the full spectrum (a canonical bin with
// 0 < kx < M stands for k and -k): A = sum |X|, P = sum |X|^2, n = bins.
// Block-local histograms in shared memory, then one atomic per shell.
// acc: per item 3 x S doubles.  Grid (x: bins, y: members).
static __global__ void k_ps_shells(Group g, const float2* canon, double* acc, int S) {
  extern __shared__ double hist[];   // 3 S
  const int gi = blockIdx.y;
  const int Nz = g.Nz, Ny = g.Nmid, M = g.M;
  const int64_t nb = (int64_t)Nz * Ny * (M + 1);
  const float2* c = canon + g.coff[gi];
  for (int i = threadIdx.x; i < 3 * S; i += blockDim.x) hist[i] = 0.0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % (M + 1));
    const int64_t r = i / (M + 1);
    const int ky = (int)(r % Ny), kz = (int)(r / Ny);
    const int s = ps_shell(kz, ky, kx, Nz, Ny);
    const double w = (kx > 0 && kx < M) ? 2.0 : 1.0;
    const double a = hypot((double)c[i].x, (double)c[i].y);
    atomicAdd(&hist[s], w * a);
    atomicAdd(&hist[S + s], w * a * a);
    atomicAdd(&hist[2 * S + s], w);
  }
  __syncthreads();
  double* dst = acc + (int64_t)g.item[gi] * 3 * S;
  for (int i = threadIdx.x; i < 3 * S; i += blockDim.x)
    if (hist[i] != 0.0) atomicAdd(&dst[i], hist[i]);
}

// 1D items: the shell of bin k <= N/2 is k itself (the signed frequencies k
// and -k), one bin pair per shell: A = w |X|, P = w |X|^2, n = w, w = 2 for
// 0 < k < N/2 and 1 at k = 0 and k = N/2.  acc: per item 3 x S doubles
// (zeroed).  Grid (x: bins, y: members).
static __global__ void k_ps_bins1(Group g, const ItemParams* prm, const float2* canon, double* acc, int S) {
  const int gi = blockIdx.y;
  const int item = g.item[gi];
  const int64_t N = prm[item].n, nb = N / 2 + 1;
  const float2* c = canon + g.coff[gi];
  double* A = acc + (int64_t)item * 3 * S;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nb; k += (int64_t)gridDim.x * blockDim.x) {
    const double w = (k == 0 || 2 * k == N) ? 1.0 : 2.0;
    const double a = hypot((double)c[k].x, (double)c[k].y);
    A[k] = w * a;
    A[S + k] = w * a * a;
    A[2 * S + k] = w;
  }
}

// d_s = (-2 sqrt2 A + sqrt(8 A^2 + 8 n rho P)) / (4 n) per shell; shell 0 (the
// mean) takes the smallest of the others.  One CTA per item.
static __global__ void k_ps_roots(double* acc, int S, const double* rho) {
  const int item = blockIdx.x;
  double* A = acc + (int64_t)item * 3 * S;
  double* P = A + S;
  double* n = A + 2 * S;
  __shared__ double smin[32];
  double mn = INFINITY;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    double d = 0.0;
    if (n[s] > 0.0) {
      d = (-2.0 * sqrt(2.0) * A[s] + sqrt(8.0 * A[s] * A[s] + 8.0 * n[s] * rho[item] * P[s])) / (4.0 * n[s]);
      if (s > 0) mn = fmin(mn, d);
    }
    A[s] = d;   // the root replaces the sum
  }
  for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  if ((threadIdx.x & 31) == 0) smin[threadIdx.x >> 5] = mn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = INFINITY;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) m = fmin(m, smin[w]);
    if (m < INFINITY) A[0] = m;
  }
}

// Bounds (Delta^Re, Delta^Im) = (d, d) of every canonical bin.
static __global__ void k_ps_write(Group g, const double* acc, int S, float2* out) {
  const int gi = blockIdx.y;
  const int Nz = g.Nz, Ny = g.Nmid, M = g.M;
  const int64_t nb = (int64_t)Nz * Ny * (M + 1);
  const double* d = acc + (int64_t)g.item[gi] * 3 * S;
  float2* o = out + g.coff[gi];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % (M + 1));
    const int64_t r = i / (M + 1);
    const float b = (float)d[ps_shell((int)(r / Ny), (int)(r % Ny), kx, Nz, Ny)];
    o[i] = make_float2(b, b);
  }
}

// 1D items: bounds (d_k, d_k) of bins k <= N/2.
static __global__ void k_ps_write1(Group g, const ItemParams* prm, const double* acc, int S, float2* out) {
  const int gi = blockIdx.y;
  const int item = g.item[gi];
  const int64_t nb = prm[item].n / 2 + 1;
  const double* d = acc + (int64_t)item * 3 * S;
  float2* o = out + g.coff[gi];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nb; k += (int64_t)gridDim.x * blockDim.x) {
    const float b = (float)d[k];
    o[k] = make_float2(b, b);
  }
}

// ----- decompression side: edits from their stored form ----------------------
// (Sec. IV-B, "Applying edits to the decompressed data")

struct ApRegion {
  const uint8_t* flags;
  const int32_t* codes;
  int64_t n;
  int* chunks;
  float q;
  float* xhat;      // spatial: the item's reconstruction (edits added in place)
  float2* dense;    // frequency: the item's canonical half spectrum (written)
};

// Nonzero components per chunk from the flag bytes.
static __global__ void k_apply_count(const ApRegion* regs) {
  const ApRegion r = regs[blockIdx.y];
  const int64_t c0 = (int64_t)blockIdx.x * kEdChunk;
  if (c0 >= r.n) return;
  const int64_t b = c0 / 8 + threadIdx.x;
  int cnt = (b * 8 < r.n) ? __popc((unsigned)r.flags[b]) : 0;
  __shared__ int s[kEdThreads / 32];
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kEdThreads / 32; ++w) t += s[w];
    r.chunks[blockIdx.x] = t;
  }
}

// Exclusive scan of the chunk counts (one CTA per region).
static __global__ void k_apply_scan(const ApRegion* regs) {
  const ApRegion r = regs[blockIdx.x];
  const int64_t nch = (r.n + kEdChunk - 1) / kEdChunk;
  __shared__ long long carry;
  __shared__ long long s[1024];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nch; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const long long v = i < nch ? r.chunks[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
      const long long add = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < nch) r.chunks[i] = (int)(carry + s[threadIdx.x] - v);
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += s[threadIdx.x];
    __syncthreads();
  }
}

// Dequantize (code * q) and place: spatial edits are added to x_hat,
// frequency edits written densely (zero where the flag is clear).
template <bool FREQ>
static __global__ void k_apply_expand(const ApRegion* regs) {
  const ApRegion r = regs[blockIdx.y];
  const int64_t c0 = (int64_t)blockIdx.x * kEdChunk;
  if (c0 >= r.n) return;
  const int64_t b = c0 / 8 + threadIdx.x;
  const unsigned byte = (b * 8 < r.n) ? r.flags[b] : 0u;
  const int cnt = __popc(byte);
  __shared__ int s[kEdThreads / 32];
  int incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if ((threadIdx.x & 31) >= (unsigned)o) incl += y;
  }
  if ((threadIdx.x & 31) == 31) s[threadIdx.x >> 5] = incl;
  __syncthreads();
  int wbase = 0;
  for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wbase += s[w];
  int64_t k = (int64_t)r.chunks[blockIdx.x] + wbase + incl - cnt;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int64_t i = b * 8 + t;
    if (i >= r.n) break;
    const bool on = (byte >> t) & 1u;
    if constexpr (FREQ) {
      r.dense[i] = on ? make_float2((float)r.codes[2 * k] * r.q, (float)r.codes[2 * k + 1] * r.q)
                      : make_float2(0.f, 0.f);
    } else if (on) {
      r.xhat[i] += (float)r.codes[k] * r.q;
    }
    k += on;
  }
}

// Canonical half spectrum -> packed layout (kx = 0 slot = A + iB with
// A, B the kx = 0 and kx = Nx/2 planes).  Grid (x: slots, y: members).
static __global__ void k_edits_pack(Group g, const float2* canon, const int64_t* coff, float2* packed) {
  const int gi = blockIdx.y;
  const int Nz = g.Nz, Ny = g.Nmid, M = g.M;
  const int64_t ns = (int64_t)Nz * Ny * M;
  const float2* c = canon + coff[gi];
  float2* o = packed + g.soff[gi];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % M);
    const int64_t r = i / M;
    if (kx) {
      o[i] = c[r * (M + 1) + kx];
    } else {
      const float2 A = c[r * (M + 1)], B = c[r * (M + 1) + M];
      o[i] = make_float2(A.x - B.y, A.y + B.x);
    }
  }
}

}  // namespace ffcz
