// bluestein.cuh -- 1D items of any length N: the DFT of Eq. 1 by Bluestein's
// chirp-z identity on a power-of-two length P >= 2N - 1 (sm_103a).
//
// With b_m = exp(i pi m^2 / N):  X_k = conj(b_k) sum_n (x_n conj(b_n)) b_{k-n},
// a circular convolution of length P with the wrapped chirp f (f[m] = b_m and
// f[P-m] = b_m for 0 <= m < N, zero between):  X = conj(b) IFFT_P(FFT_P(a) Bt)/P,
// Bt = FFT_P(f).  The inverse DFT uses the conjugate chirps; as f is even,
// FFT_P(conj f) = conj(Bt).
//
// FFT_P runs as a four-step transform over a [P1][P2] array (index
// n = P2 n1 + n2): column FFTs of length P1, the factor exp(-2 pi i n2 k1/P),
// row FFTs of length P2, leaving the spectrum in [k1][k2] order
// (k = k1 + P1 k2); the inverse walks the same steps backwards and returns to
// natural order.  Pointwise work rides on the passes:
//   row pass  : FFT along the row, times Bt (or conj Bt), IFFT along the row
//   column pass: inverse column step (twiddle, IFFT), chirp post-multiply
//               (-> X_k or x_n in natural order), the check and the clip of
//               Alg. 1, chirp pre-multiply, forward column step.
// One iteration is: row(conj Bt), column(s-clip), row(Bt), column(f-check,
// f-clip) -- four passes, like the 3D schedule.  The adjoint step
// g <- Re(IDFT(M_f DFT(M_s g))) runs the same chain with the clips replaced by
// their active-set masks (M_MASK), kept as one byte per point (1: inside the
// s-cube) and one per bin k < N (bit 0: Re inside, bit 1: Im inside) at the
// item's point offset; M_RECORD writes them while the forward is replayed.  Only k, n < N carry data;
// the rest of the P-length buffers is the zero padding of the convolution.
#pragma once
#include "passes.cuh"

namespace ffcz {

enum Op1 : int {
  OP1_ENTRY = 0,   // column: load real x, pre-multiply, forward column step
  OP1_FCLIP = 1,   // column: inverse step, X = conj(b) c / P, check, clip, pre, forward
  OP1_SCLIP = 2,   // column: inverse step, x = Re(b c)/(P N), s-clip, pre, forward
  OP1_EXIT = 3,    // column: inverse step, x, s-clip, store float32 e
  OP1_FILTER = 4,  // column: forward column step of the wrapped chirp f (Bt build)
  OP1_LOADX = 5,   // column: half spectrum X (k <= N/2) -> X_k b_k, forward column step
  OP1_STOREX = 6,  // column: inverse step, X_k = conj(b_k) c_k / P, store bins k <= N/2
  OP1_ZOUT = 7,    // column: inverse step, Z_k = conj(b_k) c_k / P (k < N), float64 to zout
  OP1_CONV = 8,    // row: FFT, times Bt, IFFT
  OP1_CONVC = 9,   // row: FFT, times conj Bt, IFFT
  OP1_FWD = 10     // row: FFT only (Bt build)
};

// Chirp b_m = exp(i pi m^2 / N) from r = m^2 mod 2N: the phase r/N is in
// [0, 2); sincospi of the part below 1 (the CUDA function is called), the
// sign flipped for the upper half.  Used once per plan to fill the tables.
template <typename T>
__device__ __forceinline__ v2<T> chirp_r(uint64_t r, uint64_t N) {
  const bool hi = r >= N;
  const uint64_t rr = hi ? r - N : r;
  T s, c;
  if constexpr (sizeof(T) == 4) sincospif((float)rr / (float)N, &s, &c);
  else sincospi((double)rr / (double)N, &s, &c);
  return hi ? mk<T>(-c, -s) : mk<T>(c, s);
}

// Chirp table b_n, n < N, of every item of a group (one launch per plan and
// precision); stored like the items' float32 data, at the item's e offset.
template <typename T>
__global__ void k1_chirp_table(Group g, const ItemParams* prm, v2<T>* tab, int half = 0) {
  const int gi = blockIdx.y;
  const int item = g.item[gi];
  if (half && !prm[item].h1) return;
  const uint64_t N = (uint64_t)prm[item].n / (half ? 2 : 1), twoN = 2 * N;
  v2<T>* out = tab + g.eoff[gi];
  for (uint64_t n = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; n < N;
       n += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r = n % twoN * (n % twoN) % twoN;
    out[n] = chirp_r<T>(r, N);
  }
}

// Column pass along n1 / k1 (length P1 = L), tile = W consecutive columns.
// The chirp of each value is read from the item's table where it is used.
template <typename T, int L, int W_ = TileW<T>::value>
__device__ __forceinline__ void k1_col_body(const Args& a, const int bx_, const int by_) {
  FFCZ_AXIS_PROLOGUE(T, L, W_, 0)
  if ((a.half1 == 1 && !p.h1) || (a.half1 == 2 && p.h1)) return;   // certification split (member-uniform)
  constexpr int NT = G_::NT, W = G_::W;
  const int P2 = a.g.M;
  const int64_t N = a.half1 == 1 ? p.n / 2 : p.n;   // transform length
  const int ntiles = P2 / W;
  const bool live = tile < ntiles;
  const int n2 = live ? tile * W + w : 0;
  const int64_t ustride = (int64_t)NT * P2;
  const v2<T>* twp = reinterpret_cast<const v2<T>*>(a.twr);      // exp(-2 pi i m / P), m < P
  const int op = a.op1;
  const uint64_t m0 = (uint64_t)j * P2 + n2, D = (uint64_t)NT * P2;
  const int64_t Pn = (int64_t)L * P2;
  const v2<T>* ctab = reinterpret_cast<const v2<T>*>(a.chirp) + a.g.eoff[gi];
  auto chirp = [&](int u) -> v2<T> {   // b_n of value u (zero past N)
    const int64_t n = (int64_t)m0 + (int64_t)u * D;
    return (live && n < N) ? ctab[n] : mk<T>(T(0), T(0));
  };
  v2<T> v[V];
  AbsMax<T> mx;
  bool bad = false;
  float ssq = 0.f;
  unsigned long long cnt = 0;
  // pointwise bounds (null: the item's scalar bounds): E_n at the item's e
  // offset, (Delta^Re, Delta^Im) of bins k <= N/2 at its half-spectrum
  // offset (bin k > N/2 takes those of N - k); the measures are then ratios
  const float* pwe = a.pw_e ? a.pw_e + a.g.eoff[gi] : nullptr;
  const float2* pwf = a.pw_f ? a.pw_f + a.g.coff[gi] : nullptr;
  if (op == OP1_ENTRY && a.half1 == 1) {
    // z_n = x_2n + i x_2n+1 (certification: measure only)
    const float* src = a.e + a.g.eoff[gi];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int64_t n = (int64_t)m0 + (int64_t)u * D;
      const bool in = live && n < N;
      const float x = in ? src[2 * n] : 0.f, y = in ? src[2 * n + 1] : 0.f;
      if ((a.mode & M_MEASURE) && in) {
        if (pwe) { mx.add((T)ratio_cert(x, pwe[2 * n])); mx.add((T)ratio_cert(y, pwe[2 * n + 1])); }
        else { mx.add((T)x); mx.add((T)y); }
        bad |= (x != x) | (y != y);
        ssq = fmaf(x, x, fmaf(y, y, ssq));
      }
      v[u] = mk<T>((T)x, (T)y);
    }
  } else if (op == OP1_ENTRY) {
    float* src = a.e + a.g.eoff[gi];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int64_t n = (int64_t)m0 + (int64_t)u * D;
      float x = (live && n < N) ? src[n] : 0.f;
      const float ebn = (pwe && live && n < N) ? pwe[n] : 1.f;
      if (a.mode & M_MEASURE) {
        mx.add(pwe ? (T)ratio_cert(x, ebn) : (T)x);
        bad |= (x != x);
        ssq = fmaf(x, x, ssq);
      }
      if ((a.mode & M_MASK) && !(live && n < N && reinterpret_cast<const uint8_t*>(a.mask)[a.g.eoff[gi] + n]))
        x = 0.f;   // adjoint: M_s of the first step
      if (a.mode & M_PRECLIP) {
        const float cx = clampT(x, p.Esf * ebn);
        cnt += (cx != x);
        if (a.ed_s && live && n < N && cx != x) atomicAdd(a.ed_s + a.g.eoff[gi] + n, cx - x);   // S += eps' - eps
        x = cx;
        if (live && n < N) src[n] = x;
      }
      v[u] = mk<T>((T)x, T(0));
    }
  } else if (op == OP1_LOADX) {
    // X_k b_k from the item's half spectrum (bin k > N/2 is conj X_{N-k})
    const float2* hx = a.ed_f + a.g.coff[gi];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int64_t k = (int64_t)m0 + (int64_t)u * D;
      v2<T> X = mk<T>(T(0), T(0));
      if (live && k < N) {
        const float2 h = hx[k <= N / 2 ? k : N - k];
        X = mk<T>((T)h.x, k <= N / 2 ? (T)h.y : -(T)h.y);
      }
      v[u] = cmul<T>(X, chirp(u));
    }
  } else if (op != OP1_FILTER) {
    const v2<T>* in = pick<T>(a, a.sel_in, t_it) + a.g.soff[gi] + m0;
#pragma unroll
    for (int u = 0; u < V; ++u) v[u] = in[u * ustride];
  }
  load_tables<T>(s_tw, a.tw, L, nullptr, nullptr, 0);

  if (op == OP1_FILTER) {
    // wrapped chirp: f[m] = b_m for m < N, f[m] = b_{P-m} for 0 < P - m < N
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int64_t m = (int64_t)m0 + (int64_t)u * D, q = Pn - m;
      v2<T> f = mk<T>(T(0), T(0));
      if (live && m < N) f = ctab[m];
      else if (live && q < N) f = ctab[q];
      v[u] = f;
    }
  } else if (op == OP1_ENTRY) {
#pragma unroll
    for (int u = 0; u < V; ++u) v[u] = cmulc<T>(v[u], chirp(u));   // a_n = x_n conj(b_n)
    if (a.mode & (M_MEASURE | M_PRECLIP)) {
      // at most 2V <= 64 float32 squares: relative error of the sum < 2^-18
      Red rr{live ? mx.dbits(bad) : 0ull, live ? (double)ssq * (1.0 + 0x1p-17) : 0.0, live ? cnt : 0ull};
      block_reduce(rr, s_red);
      if (threadIdx.x == 0) {
        if (a.mode & M_MEASURE) {
          atomicMax(&st.emaxbits, rr.vbits);
          atomicAdd(&st.sumsq, rr.sum);
        }
        if ((a.mode & M_PRECLIP) && rr.cnt) atomicAdd(&st.act_s, rr.cnt);
      }
    }
  } else if (op != OP1_LOADX) {
    // inverse column step: conj twiddle, IFFT along k1 -> c[n1][n2] * P
#pragma unroll
    for (int u = 0; u < V; ++u) v[u] = cmulc<T>(v[u], twp[(j + u * NT) * n2]);
    fft_pencil<T, L, +1>(v, j, s_tw, tl);
    const bool count = (a.mode & M_COUNT) != 0;
    if (op == OP1_ZOUT) {   // Z_k, k < N (certification of even lengths)
      const T invP = T(1) / (T)Pn;
      v2<T>* zo = reinterpret_cast<v2<T>*>(a.zout) + a.g.soff[gi];
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const int64_t k = (int64_t)m0 + (int64_t)u * D;
        if (!(live && k < N)) continue;
        const v2<T> Z = cmulc<T>(v[u], chirp(u));
        zo[k] = mk<T>(Z.x * invP, Z.y * invP);
      }
      return;
    }
    if (op == OP1_STOREX) {   // the item's half spectrum into ed_f at its canonical offset
      const T invP = T(1) / (T)Pn;
      float2* hx = a.ed_f + a.g.coff[gi];
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const int64_t k = (int64_t)m0 + (int64_t)u * D;
        if (!(live && k <= N / 2)) continue;
        const v2<T> X = cmulc<T>(v[u], chirp(u));
        hx[k] = make_float2((float)(X.x * invP), (float)(X.y * invP));
      }
      return;
    }
    if (op == OP1_FCLIP) {
      const T invP = T(1) / (T)Pn;   // exact: P is a power of two
      const T Ds = sizeof(T) == 4 ? (T)p.Dsf : (T)p.Ds;
      const bool clip = (a.mode & M_CLIP) != 0;
      // edits: bins k <= N/2 (the half spectrum); clips at the max_iters
      // check are not recorded, and a marginal one (at most the stopping
      // threshold, from min_iters on) is remembered for the loop's end
      const bool rec_f = clip && a.ed_t != nullptr && t_it < p.max_iters;
      const bool may_stop = t_it >= p.min_iters;
      const T thr = sizeof(T) == 4 ? (T)p.thrf : (T)p.thr;
      // Dykstra / Douglas-Rachford: residual r of the previous frequency
      // projection per bin k < N (zero before the first one); y = P_F'(X + r),
      // r <- X + r - y, output y (Dykstra) or y - r (Douglas-Rachford)
      const bool res = clip && (a.pv == PV_DYKSTRA || a.pv == PV_DR);
      float2* rr = res ? a.pv_r + a.g.eoff[gi] : nullptr;
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const int64_t k = (int64_t)m0 + (int64_t)u * D;
        const bool in_range = live && k < N;
        const v2<T> bk = chirp(u);
        v2<T> X = cmulc<T>(v[u], bk);            // X_k = conj(b_k) c_k / P
        X = mk<T>(X.x * invP, X.y * invP);
        T qx = T(1), qy = T(1);
        if (pwf && in_range) {
          const float2 q = pwf[k <= N / 2 ? k : N - k];
          qx = (T)q.x; qy = (T)q.y;
        }
        if (in_range) {
          if (pwf) { mx.add(ratioT(X.x, qx)); mx.add(ratioT(X.y, qy)); }
          else { mx.add(X.x); mx.add(X.y); }
          bad |= (X.x != X.x) | (X.y != X.y);
        }
        uint8_t* fmk = (a.mode & (M_MASK | M_RECORD))
                           ? reinterpret_cast<uint8_t*>(a.mask + (int64_t)t_it * a.mask_step) + a.g.eoff[gi]
                           : nullptr;
        if (a.mode & M_MASK) {   // adjoint: M_f
          const unsigned b = in_range ? fmk[k] : 0u;
          X = mk<T>((b & 1u) ? X.x : T(0), (b & 2u) ? X.y : T(0));
        } else if (res) {
          const float2 r0 = (t_it >= 1 && in_range) ? rr[k] : make_float2(0.f, 0.f);
          const T x = X.x + (T)r0.x, y = X.y + (T)r0.y;
          const T cx = clampT(x, Ds), cy = clampT(y, Ds);
          if (count && in_range) cnt += (cx != x) + (cy != y);
          const T rx = x - cx, ry = y - cy;
          if (in_range) rr[k] = make_float2((float)rx, (float)ry);
          X = a.pv == PV_DYKSTRA ? mk<T>(cx, cy) : mk<T>(cx - rx, cy - ry);
        } else if (clip) {
          const T cx = clampT(X.x, Ds * qx), cy = clampT(X.y, Ds * qy);
          if (count && in_range) cnt += (cx != X.x) + (cy != X.y);
          if (rec_f && in_range && k <= N / 2) {
            const T big = pwf ? fmax(ratioT(fabs(X.x), qx), ratioT(fabs(X.y), qy)) : fmax(fabs(X.x), fabs(X.y));
            record_f(a, a.g.coff[gi] + k, (float)(cx - X.x), (float)(cy - X.y), t_it, may_stop && big <= thr);
          }
          if ((a.mode & M_RECORD) && in_range) fmk[k] = (uint8_t)((cx == X.x) | ((cy == X.y) << 1));
          X = mk<T>(cx, cy);
        }
        v[u] = in_range ? cmul<T>(X, bk) : mk<T>(T(0), T(0));   // pre: X'_k b_k
      }
      unsigned long long vb = mx.dbits(bad);
      block_max_count(vb, cnt, count, s_red);
      if (threadIdx.x == 0) {
        atomicMax(&st.vbits, vb);
        if (cnt) atomicAdd(&st.act_f, cnt);
      }
      if (a.mode & M_NOWRITE) return;
    } else {
      const T inv_pn = sizeof(T) == 4 ? (T)p.inv_pnf : (T)p.inv_pn;
      const T Es = sizeof(T) == 4 ? (T)p.Esf : (T)p.Es;
      float* eo = a.e + a.g.eoff[gi];
      float* eo_s = a.ed_s ? a.ed_s + a.g.eoff[gi] : nullptr;   // spatial edits S += eps' - eps
      // Dykstra's q / ADMM's scaled dual u, one buffer per iteration parity
      // (zero before the second s-projection); ADMM checks a_t (the input)
      // against the s-cube
      const int pv = a.pv;
      const bool qv = (pv == PV_DYKSTRA || pv == PV_ADMM) && (a.mode & M_CLIP);
      const float* q_in = (pv == PV_DYKSTRA || pv == PV_ADMM) && t_it >= 2 ? a.pv_q[(t_it - 1) & 1] + a.g.eoff[gi]
                                                                            : nullptr;
      float* q_out = qv && op == OP1_SCLIP ? a.pv_q[t_it & 1] + a.g.eoff[gi] : nullptr;
      AbsMax<T> svm;
      // checkpoints of e_t for t = 0, m, 2m, ... below the item's K
      float* ckp = ((a.mode & M_CKPT) && a.ckpt_every > 0 && (t_it % a.ckpt_every) == 0 && t_it < p.max_iters)
                       ? a.ckpt + (int64_t)(t_it / a.ckpt_every) * a.ckpt_stride + a.g.eoff[gi]
                       : nullptr;
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const int64_t n = (int64_t)m0 + (int64_t)u * D;
        const bool in_range = live && n < N;
        const v2<T> bn = chirp(u);
        T x = (bn.x * v[u].x - bn.y * v[u].y) * inv_pn;   // Re(b_n c'_n) / (P N)
        const float ebn = (pwe && in_range) ? pwe[n] : 1.f;
        if (qv && op == OP1_SCLIP) {
          const T q0 = (q_in && in_range) ? (T)q_in[n] : T(0);
          if (pv == PV_ADMM && in_range) svm.add(x);
          const T wv = x + q0, c = clampT(wv, Es);
          if (count && in_range) cnt += (c != wv);
          if (in_range) q_out[n] = (float)(wv - c);
          x = pv == PV_DYKSTRA ? c : c - (wv - c);   // ADMM forwards b - u
        } else if (op == OP1_EXIT && pv == PV_DYKSTRA && q_in && in_range) {
          x += (T)q_in[n];   // x_t = P_S'(y_{t-1} + q_{t-1})
        }
        if ((a.mode & M_MASK) && op == OP1_SCLIP) {   // adjoint: M_s
          if (!(in_range && reinterpret_cast<const uint8_t*>(a.mask)[a.g.eoff[gi] + n])) x = T(0);
        } else if ((a.mode & M_CLIP) && !(qv && op == OP1_SCLIP)) {
          const T cx = clampT(x, Es * (T)ebn);
          if (count && in_range) cnt += (cx != x);
          if (op == OP1_SCLIP && a.ed_s && in_range && cx != x) atomicAdd(eo_s + n, (float)(cx - x));
          if (op == OP1_SCLIP && (a.mode & M_RECORD) && in_range)
            reinterpret_cast<uint8_t*>(a.mask + (int64_t)t_it * a.mask_step)[a.g.eoff[gi] + n] = (uint8_t)(cx == x);
          x = cx;
        }
        if (op == OP1_SCLIP && ckp && in_range) ckp[n] = (float)x;   // checkpoint e_t
        if (op == OP1_EXIT) {
          if (in_range && (a.mode & M_ACC)) eo[n] += (float)x;   // decompression side: x_hat += IDFT(F)
          else if (in_range) eo[n] = (a.mode & M_CLIP) ? clampT((float)x, p.Esf * ebn) : (float)x;
        } else {
          v[u] = in_range ? cmulc<T>(mk<T>(x, T(0)), bn) : mk<T>(T(0), T(0));   // x_n conj(b_n)
        }
      }
      if (op == OP1_EXIT) return;
      if (count || (qv && pv == PV_ADMM)) {
        // ADMM: max |a_t| over the CTA's points (NaN -> +inf)
        unsigned long long vb = (qv && pv == PV_ADMM) ? svm.dbits(svm.val() != svm.val()) : 0ull;
        block_max_count(vb, cnt, count, s_red);
        if (threadIdx.x == 0) {
          if (qv && pv == PV_ADMM) atomicMax(&st.svbits, vb);
          if (cnt) atomicAdd(&st.act_s, cnt);
        }
      }
    }
  }
  // forward column step: FFT along n1, twiddle exp(-2 pi i n2 k1 / P)
  fft_pencil<T, L, -1>(v, j, s_tw, tl);
  if (live) {
    v2<T>* out = pick<T>(a, a.sel_out, t_it) + a.g.soff[gi] + m0;
#pragma unroll
    for (int u = 0; u < V; ++u) out[u * ustride] = cmul<T>(v[u], twp[(j + u * NT) * n2]);
  }
}
template <typename T, int L, int W_ = TileW<T>::value>
__global__ void __launch_bounds__(Geo<T, L, W_>::NTHR, Geo<T, L, W_>::MINB)
k1_col(Args a) {
  k1_col_body<T, L, W_>(a, (int)blockIdx.x, (int)blockIdx.y);
}

// Row pass along n2 / k2 (length P2 = L), tile = W consecutive rows.
template <typename T, int L, int W_ = TileW<T>::value>
__device__ __forceinline__ void k1_row_body(const Args& a, const int bx_, const int by_) {
  FFCZ_AXIS_PROLOGUE(T, L, W_, 0)
  if ((a.half1 == 1 && !p.h1) || (a.half1 == 2 && p.h1)) return;   // certification split (member-uniform)
  constexpr int NT = G_::NT;
  const int P1 = a.g.Nz;
  const int prow = tile * G_::W + w;
  const bool live = prow < P1;
  const int row = live ? prow : 0;
  const v2<T>* in = pick<T>(a, a.sel_in, t_it) + a.g.soff[gi] + (int64_t)row * L + j;
  v2<T> v[V];
#pragma unroll
  for (int u = 0; u < V; ++u) v[u] = in[u * NT];
  load_tables<T>(s_tw, a.tw, L, nullptr, nullptr, 0);
  fft_pencil<T, L, -1>(v, j, s_tw, tl);
  if (a.op1 != OP1_FWD) {
    const v2<T>* bt = reinterpret_cast<const v2<T>*>(a.bt) + a.g.soff[gi] + (int64_t)row * L + j;
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const v2<T> f = bt[u * NT];
      v[u] = a.op1 == OP1_CONVC ? cmulc<T>(v[u], f) : cmul<T>(v[u], f);
    }
    fft_pencil<T, L, +1>(v, j, s_tw, tl);
  }
  if (live) {
    v2<T>* out = pick<T>(a, a.sel_out, t_it) + a.g.soff[gi] + (int64_t)row * L + j;
#pragma unroll
    for (int u = 0; u < V; ++u) out[u * NT] = v[u];
  }
}
template <typename T, int L, int W_ = TileW<T>::value>
__global__ void __launch_bounds__(Geo<T, L, W_>::NTHR, Geo<T, L, W_>::MINB)
k1_row(Args a) {
  k1_row_body<T, L, W_>(a, (int)blockIdx.x, (int)blockIdx.y);
}

// Twiddles W_N^k = exp(-2 pi i k / N), k <= N/2, of the members certified
// through the N/2-point transform (at the canonical offset; the CUDA
// function is called).  Grid (x: any, y: members).
__global__ void k1_rtw(Group g, const ItemParams* prm, double2* W) {
  const int gi = blockIdx.y;
  const int item = g.item[gi];
  if (!prm[item].h1) return;
  const int64_t N = prm[item].n;
  double2* w = W + g.coff[gi];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= N / 2; k += (int64_t)gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi((double)(2 * k) / (double)N, &sn, &cs);
    w[k] = make_double2(cs, -sn);
  }
}

// Certification of even lengths: from Z = DFT_{N/2}(x_2n + i x_2n+1), the
// spectrum of the real signal X_k = (A - i W_N^k B) / 2 with
// A = Z_k + conj Z_{N/2-k}, B = Z_k - conj Z_{N/2-k} (indices mod N/2), for
// k <= N/2 (the rest mirrors them), and the violation max (ratios with
// pointwise bounds, NaN -> +inf) into the item's vbits.  Grid (x: any,
// y: members), 256 threads.
__global__ void __launch_bounds__(256) k1_rpost(Group g, const ItemParams* prm, ItemState* st, int pred,
                                                const double2* Z, const double2* W, const float2* pwf) {
  const int gi = blockIdx.y;
  const int item = g.item[gi];
  const ItemParams& p = prm[item];
  ItemState& s = st[item];
  if (!p.h1 || !pred_ok(pred, s, p)) return;
  const int64_t N = p.n, H = N / 2;
  const double2* z = Z + g.soff[gi];
  const double2* w = W + g.coff[gi];
  const float2* q = pwf ? pwf + g.coff[gi] : nullptr;
  AbsMax<double> mx;
  bool bad = false;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= H; k += (int64_t)gridDim.x * blockDim.x) {
    const double2 zk = z[k == H ? 0 : k], zm = z[k == 0 ? 0 : H - k];
    const double ar = zk.x + zm.x, ai = zk.y - zm.y, br = zk.x - zm.x, bi = zk.y + zm.y;
    const double2 wk = w[k];
    const double pr = wk.x * br - wk.y * bi, pi = wk.x * bi + wk.y * br;   // W B
    const double xr = 0.5 * (ar + pi), xi = 0.5 * (ai - pr);               // (A - i W B) / 2
    if (q) { mx.add(xr / (double)q[k].x); mx.add(xi / (double)q[k].y); }
    else { mx.add(xr); mx.add(xi); }
    bad |= (xr != xr) | (xi != xi);
  }
  __shared__ unsigned long long s_red[128];
  unsigned long long vb = mx.dbits(bad), c = 0ull;
  block_max_count(vb, c, false, s_red);
  if (threadIdx.x == 0) atomicMax(&s.vbits, vb);
}

}  // namespace ffcz
