// Vector kernels of one Lanczos step (Eq. 13), FP64.
//
// Step j of every start vector b in a sub-batch (w already holds
// C q_j - beta_j q_{j-1} from the contraction epilogue):
//   alpha_j = q_j . w          (per-tile partials summed in fixed order)
//   w <- w - alpha_j q_j
//   full reorthogonalisation against the stored basis q_0..q_j by classical
//   Gram-Schmidt: h = Q^T w, w <- w - Q h (once, or twice)
//   beta_{j+1} = ||w||; stop when beta_{j+1} <= tol * max|alpha|
//   q_{j+1} = w / beta_{j+1};  xh = bf16(Delta^1/2 q_{j+1})
//
// Every block owns one chunk of VEC_CHUNK pair elements of one vector; each
// warp owns 256 consecutive elements, each lane four double2 of them.  All
// cross-block sums go through per-chunk partials reduced in a fixed order,
// so results do not depend on scheduling.
#include "lgw_internal.cuh"

namespace lgw {

__device__ __forceinline__ int elem_base(int chunk) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  return chunk * VEC_CHUNK + wid * 256 + 2 * lane;
}

__device__ __forceinline__ bool vec_live(const VecCtx &c, int b, int j) {
  return b < c.nvec && c.k_eff[c.vec0 + b] > j;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic for the float-pair vector passes (Dekker 1971,
// Knuth's TwoSum): a value is hi + lo with |lo| <= ulp(hi) / 2, 48 bits.
// These passes leave most issue slots idle while GB300's FP64 pipe (2 lanes
// per SM clock) bounds them, so FP32-pipe arithmetic costs nothing there.
// Products drop lo * lo (relative error about 2^-46).
// ---------------------------------------------------------------------------
struct dfl {
  float h, l;
};
__device__ __forceinline__ dfl df_fast(float a, float b) {   // |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return df_fast(p, e);
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {   // accurate under cancellation
  dfl s = df_two_sum(a.h, b.h);
  const dfl t = df_two_sum(a.l, b.l);
  s = df_fast(s.h, __fadd_rn(s.l, t.h));
  return df_fast(s.h, __fadd_rn(s.l, t.l));
}
__device__ __forceinline__ dfl df_add_f(dfl a, float b) {
  const dfl s = df_two_sum(a.h, b);
  return df_fast(s.h, __fadd_rn(s.l, a.l));
}
__device__ __forceinline__ dfl df_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
// (sh, sl) += a . b, TwoProd with the cross terms and TwoSum
__device__ __forceinline__ void df_dot_acc(float &sh, float &sl, dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  const dfl s = df_two_sum(sh, p);
  sh = s.h;
  sl = __fadd_rn(__fadd_rn(sl, s.l), e);
}
// hi and lo halves of a float-pair slot [Bs][N] (hi, then lo)
__device__ __forceinline__ float *pair_hi(double *slot, const VecCtx &c) {
  return reinterpret_cast<float *>(slot);
}
__device__ __forceinline__ float *pair_lo(double *slot, const VecCtx &c) {
  return reinterpret_cast<float *>(slot) + (size_t)c.Bs * c.N;
}

// Partial dot products of the thread's eight elements of w with basis rows
// 0..nrows-1 of vector b; one partial per (row, chunk) after a warp
// transposed reduction and a fixed-order sum over the eight warps.
__device__ void dots_rows(const VecCtx &c, int nrows, int b, int chunk, const double (&wr)[8],
                          double (*sred)[32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int e0 = elem_base(chunk);
  const size_t voff = (size_t)b * c.N;
  for (int r0 = 0; r0 < nrows; r0 += 32) {
    double acc[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      acc[r] = 0.0;
      if (r0 + r < nrows) {
        const double *qrow = slot_ptr(c, r0 + r) + voff;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = e0 + u * 64;
          if (e < c.N) {
            const double2 q2 = *reinterpret_cast<const double2 *>(qrow + e);
            acc[r] = fma(q2.x, wr[2 * u], acc[r]);
            acc[r] = fma(q2.y, wr[2 * u + 1], acc[r]);
          }
        }
      }
    }
    warp_transpose_sum32(acc);
    sred[wid][lane] = acc[0];
    __syncthreads();
    if (wid == 0) {
      double s = 0.0;
#pragma unroll
      for (int w8 = 0; w8 < VEC_THREADS / 32; ++w8) s += sred[w8][lane];
      if (r0 + lane < nrows)
        c.dot_part[((size_t)b * c.nchunks + chunk) * c.kmax1 + r0 + lane] = s;
    }
    __syncthreads();
  }
}

// Tensor-core path without reorthogonalisation: the contraction leaves
// ucd = c_K Delta^1/2 (L y) in FP32 (store-only epilogue); here, in FP64,
//   w = Delta^2 q_j + ucd - beta_j q_{j-1}
// and per-chunk partials of alpha_j = q_j . w (alpha_part[chunk][b]).
__device__ __forceinline__ void assemble_w_chunk(const VecCtx &c, int j,
                                                 const float *__restrict__ ucd, int chunk,
                                                 int b) {
  __shared__ double red[VEC_THREADS / 32];
  if (!vec_live(c, b, j)) return;
  const size_t voff = (size_t)b * c.N;
  const double bj = c.betaj[b];
  const int e0 = elem_base(chunk);
  if (c.pair) {
    // the same in double-float on float pairs (w = (Delta^2 q + ucd) - beta_j q_{j-1})
    const float *qh = pair_hi(slot_ptr(c, j), c) + voff, *ql = pair_lo(slot_ptr(c, j), c) + voff;
    const float *ph = j > 0 ? pair_hi(slot_ptr(c, j - 1), c) + voff : nullptr;
    const float *pl = j > 0 ? pair_lo(slot_ptr(c, j - 1), c) + voff : nullptr;
    float *wh = pair_hi(c.w, c) + voff, *wl = pair_lo(c.w, c) + voff;
    const dfl nbj = (j > 0 && c.nbeta_f) ? dfl{c.nbeta_f[b].x, c.nbeta_f[b].y} : df_from(-bj);
    float sh = 0.f, sl = 0.f;
#pragma unroll
    for (int u4 = 0; u4 < 4; ++u4) {
      const int e = e0 + u4 * 64;
      if (e >= c.N) continue;
      const float2 a2 = *reinterpret_cast<const float2 *>(qh + e);
      const float2 b2 = *reinterpret_cast<const float2 *>(ql + e);
      const float2 v2 = *reinterpret_cast<const float2 *>(ucd + kblk_f32(b, e, c.Bs));
      const float2 dh = *reinterpret_cast<const float2 *>(c.d2f + e);
      const float2 dl = *reinterpret_cast<const float2 *>(c.d2lo + e);
      float2 p2 = make_float2(0.f, 0.f), r2 = p2;
      if (ph != nullptr) {
        p2 = *reinterpret_cast<const float2 *>(ph + e);
        r2 = *reinterpret_cast<const float2 *>(pl + e);
      }
      const dfl q0{a2.x, b2.x}, q1{a2.y, b2.y};
      dfl w0 = df_add_f(df_mul({dh.x, dl.x}, q0), v2.x);
      dfl w1 = df_add_f(df_mul({dh.y, dl.y}, q1), v2.y);
      if (ph != nullptr) {
        w0 = df_add(w0, df_mul(nbj, {p2.x, r2.x}));
        w1 = df_add(w1, df_mul(nbj, {p2.y, r2.y}));
      }
      *reinterpret_cast<float2 *>(wh + e) = make_float2(w0.h, w1.h);
      *reinterpret_cast<float2 *>(wl + e) = make_float2(w0.l, w1.l);
      df_dot_acc(sh, sl, q0, w0);
      df_dot_acc(sh, sl, q1, w1);
    }
    const double ap = block_sum_to0((double)sh + (double)sl, red);
    if (threadIdx.x == 0) c.alpha_part[(size_t)chunk * c.Bs + b] = ap;
    return;
  }
  const double *q = slot_ptr(c, j) + voff;
  const double *qp = j > 0 ? slot_ptr(c, j - 1) + voff : nullptr;
  double *w = c.w + voff;
  double ap = 0.0;
#pragma unroll
  for (int u4 = 0; u4 < 4; ++u4) {
    const int e = e0 + u4 * 64;
    if (e >= c.N) continue;
    const double2 q2 = *reinterpret_cast<const double2 *>(q + e);
    const float2 v2 = *reinterpret_cast<const float2 *>(ucd + kblk_f32(b, e, c.Bs));
    double2 w2;
    w2.x = fma(c.Delta2[e], q2.x, (double)v2.x);
    w2.y = fma(c.Delta2[e + 1], q2.y, (double)v2.y);
    if (qp != nullptr) {
      const double2 p2 = *reinterpret_cast<const double2 *>(qp + e);
      w2.x = fma(-bj, p2.x, w2.x);
      w2.y = fma(-bj, p2.y, w2.y);
    }
    *reinterpret_cast<double2 *>(w + e) = w2;
    ap = fma(q2.x, w2.x, fma(q2.y, w2.y, ap));
  }
  ap = block_sum_to0(ap, red);
  if (threadIdx.x == 0) c.alpha_part[(size_t)chunk * c.Bs + b] = ap;
}

// A block takes c.cpb consecutive chunks of one vector (each with its own
// partial, so the results do not depend on cpb).  With cpb = 1 this form of
// the passes measured faster than one chunk per kernel body (the large
// system's normalisation: 15.5 -> 9.4 ms per step, bit-identical).
__device__ __forceinline__ int cpb_of(const VecCtx &c) { return c.cpb > 1 ? c.cpb : 1; }

__global__ void __launch_bounds__(VEC_THREADS, 8) k_assemble_w(VecCtx c, int j,
                                                           const float *__restrict__ ucd) {
  const int n = cpb_of(c), c0 = blockIdx.x * n, c1 = min(c.nchunks, c0 + n);
  for (int chunk = c0; chunk < c1; ++chunk) assemble_w_chunk(c, j, ucd, chunk, blockIdx.y);
}

// alpha_j = q_j . w from the n_mt epilogue partials alpha_part[t][b], one
// warp per vector in fixed order: the recorded coefficient and amax, read
// back by every block of the axpy pass (which would otherwise each repeat
// the n_mt strided loads: 12500 of them per block at N_vc 1.6M).
__global__ void k_alpha_reduce(VecCtx c, int j) {
  const int b = blockIdx.x, lane = threadIdx.x;
  if (!vec_live(c, b, j)) return;
  double s = 0.0;
  for (int t = lane; t < c.n_mt; t += 32) s += c.alpha_part[(size_t)t * c.Bs + b];
  s = warp_sum(s);
  if (lane == 0) {
    c.alpha[(size_t)(c.vec0 + b) * c.k + j] = s;
    c.amax[b] = fmax(c.amax[b], fabs(s));
    if (c.nalpha_f) {
      const dfl n = df_from(-s);
      c.nalpha_f[b] = make_float2(n.h, n.l);
    }
  }
}

// w -= alpha_j q_j, ||w||^2 partials, and (DOTS: with reorthogonalisation)
// the first-pass dot products.  Without them the kernel needs a quarter of
// the registers, so four times the warps stay resident on the FP64 pipe.
template <bool DOTS>
__device__ __forceinline__ void alpha_axpy_chunk(const VecCtx &c, int j, int chunk, int b) {
  __shared__ double red[VEC_THREADS / 32];
  __shared__ double sred[DOTS ? VEC_THREADS / 32 : 1][32];
  if (!vec_live(c, b, j)) return;
  const double alpha = c.alpha[(size_t)(c.vec0 + b) * c.k + j];
  const size_t voff = (size_t)b * c.N;
  const int e0 = elem_base(chunk);
  if constexpr (!DOTS) {
    if (c.pair) {
      const float *qh = pair_hi(slot_ptr(c, j), c) + voff;
      const float *ql = pair_lo(slot_ptr(c, j), c) + voff;
      float *wh = pair_hi(c.w, c) + voff, *wl = pair_lo(c.w, c) + voff;
      const dfl nal = c.nalpha_f ? dfl{c.nalpha_f[b].x, c.nalpha_f[b].y} : df_from(-alpha);
      float sh = 0.f, sl = 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * 64;
        if (e >= c.N) continue;
        const float2 a2 = *reinterpret_cast<const float2 *>(qh + e);
        const float2 b2 = *reinterpret_cast<const float2 *>(ql + e);
        const float2 x2 = *reinterpret_cast<const float2 *>(wh + e);
        const float2 y2 = *reinterpret_cast<const float2 *>(wl + e);
        const dfl w0 = df_add({x2.x, y2.x}, df_mul(nal, {a2.x, b2.x}));
        const dfl w1 = df_add({x2.y, y2.y}, df_mul(nal, {a2.y, b2.y}));
        *reinterpret_cast<float2 *>(wh + e) = make_float2(w0.h, w1.h);
        *reinterpret_cast<float2 *>(wl + e) = make_float2(w0.l, w1.l);
        df_dot_acc(sh, sl, w0, w0);
        df_dot_acc(sh, sl, w1, w1);
      }
      const double nrm = block_sum_to0((double)sh + (double)sl, red);
      if (threadIdx.x == 0) c.norm_a[(size_t)b * c.nchunks + chunk] = nrm;
      return;
    }
  }
  const double *q = slot_ptr(c, j) + voff;
  double *w = c.w + voff;
  double wr[8];
  double nrm = 0.0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    double2 w2 = make_double2(0.0, 0.0);
    if (e < c.N) {
      const double2 q2 = *reinterpret_cast<const double2 *>(q + e);
      w2 = *reinterpret_cast<const double2 *>(w + e);
      w2.x = fma(-alpha, q2.x, w2.x);
      w2.y = fma(-alpha, q2.y, w2.y);
      *reinterpret_cast<double2 *>(w + e) = w2;
    }
    wr[2 * u] = w2.x;
    wr[2 * u + 1] = w2.y;
    nrm = fma(w2.x, w2.x, fma(w2.y, w2.y, nrm));
  }
  nrm = block_sum(nrm, red);
  if (threadIdx.x == 0) c.norm_a[(size_t)b * c.nchunks + chunk] = nrm;
  if constexpr (DOTS) dots_rows(c, j + 1, b, chunk, wr, sred);
}

template <bool DOTS>
__global__ void __launch_bounds__(VEC_THREADS) k_alpha_axpy(VecCtx c, int j) {
  const int n = cpb_of(c), c0 = blockIdx.x * n, c1 = min(c.nchunks, c0 + n);
  for (int chunk = c0; chunk < c1; ++chunk) alpha_axpy_chunk<DOTS>(c, j, chunk, blockIdx.y);
}

// Second-pass dot products of the current w with rows 0..j.
__global__ void __launch_bounds__(VEC_THREADS) k_dots(VecCtx c, int j) {
  __shared__ double sred[VEC_THREADS / 32][32];
  const int chunk = blockIdx.x, b = blockIdx.y;
  if (!vec_live(c, b, j) || !c.flag2[b]) return;
  const double *w = c.w + (size_t)b * c.N;
  const int e0 = elem_base(chunk);
  double wr[8];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    double2 w2 = make_double2(0.0, 0.0);
    if (e < c.N) w2 = *reinterpret_cast<const double2 *>(w + e);
    wr[2 * u] = w2.x;
    wr[2 * u + 1] = w2.y;
  }
  dots_rows(c, j + 1, b, chunk, wr, sred);
}

// h[b][i] = sum over chunks of the dot partials, fixed order.
__global__ void k_reduce_dots(VecCtx c, int j, int pass) {
  const int b = blockIdx.x;
  if (!vec_live(c, b, j)) return;
  if (pass == 2 && !c.flag2[b]) return;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const double *p = c.dot_part + (size_t)b * c.nchunks * c.kmax1 + i;
    double s = 0.0;
    for (int ch = 0; ch < c.nchunks; ++ch) s += p[(size_t)ch * c.kmax1];
    c.h[(size_t)b * c.kmax1 + i] = s;
  }
}

// w <- w - sum_i h_i q_i over rows 0..j and ||w||^2 partials.
__global__ void __launch_bounds__(VEC_THREADS) k_update(VecCtx c, int j, int pass) {
  extern __shared__ double hs[];
  __shared__ double red[VEC_THREADS / 32];
  const int chunk = blockIdx.x, b = blockIdx.y;
  if (!vec_live(c, b, j)) return;
  if (pass == 2 && !c.flag2[b]) return;
  for (int i = threadIdx.x; i <= j; i += VEC_THREADS) hs[i] = c.h[(size_t)b * c.kmax1 + i];
  __syncthreads();
  const size_t voff = (size_t)b * c.N;
  double *w = c.w + voff;
  const int e0 = elem_base(chunk);
  double2 wv[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    wv[u] = (e < c.N) ? *reinterpret_cast<const double2 *>(w + e) : make_double2(0.0, 0.0);
  }
  for (int i = 0; i <= j; ++i) {
    const double hi = hs[i];
    const double *qrow = slot_ptr(c, i) + voff;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * 64;
      if (e < c.N) {
        const double2 q2 = *reinterpret_cast<const double2 *>(qrow + e);
        wv[u].x = fma(-hi, q2.x, wv[u].x);
        wv[u].y = fma(-hi, q2.y, wv[u].y);
      }
    }
  }
  double nrm = 0.0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    if (e < c.N) *reinterpret_cast<double2 *>(w + e) = wv[u];
    nrm = fma(wv[u].x, wv[u].x, fma(wv[u].y, wv[u].y, nrm));
  }
  nrm = block_sum(nrm, red);
  if (threadIdx.x == 0) (pass == 1 ? c.norm_b : c.norm_c)[(size_t)b * c.nchunks + chunk] = nrm;
}

// Second Gram-Schmidt pass: always (CGS2), or where the first pass removed
// more than half of ||w||^2 (the 1/sqrt(2) norm criterion).
__global__ void k_second_pass_decide(VecCtx c, int j) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= c.Bs) return;
  int f = 0;
  if (vec_live(c, b, j)) {
    if (c.reorth == LGW_REORTH_CGS2) {
      f = 1;
    } else {
      double na = 0.0, nb = 0.0;
      for (int ch = 0; ch < c.nchunks; ++ch) {
        na += c.norm_a[(size_t)b * c.nchunks + ch];
        nb += c.norm_b[(size_t)b * c.nchunks + ch];
      }
      f = nb < 0.5 * na;
      if (f) atomicAdd(c.n_second, 1);
    }
  }
  c.flag2[b] = f;
}

// beta_{j+1} = ||w|| from the chosen per-chunk partials (one warp per
// vector, fixed order), the breakdown test, and 1/beta (0 when the vector
// stops or is not live) for k_normalize.
__global__ void k_beta_vec(VecCtx c, int j) {
  const int b = blockIdx.x, lane = threadIdx.x;
  const int v = c.vec0 + b;
  double inv = 0.0;
  if (b < c.nvec && c.k_eff[v] > j) {
    const double *np = c.norm_a;
    if (c.reorth != LGW_REORTH_NONE) np = c.flag2[b] ? c.norm_c : c.norm_b;
    double s = 0.0;
    for (int ch = lane; ch < c.nchunks; ch += 32) s += np[(size_t)b * c.nchunks + ch];
    s = warp_sum(s);
    const double beta = sqrt(s);
    const bool stop = !(beta > c.tol * c.amax[b]);
    if (lane == 0) {
      c.beta[(size_t)v * c.k + j] = beta;
      c.betaj[b] = beta;
      if (c.nbeta_f) {
        const dfl n = df_from(-beta);
        c.nbeta_f[b] = make_float2(n.h, n.l);
      }
      if (stop) c.k_eff[v] = j + 1;
    }
    inv = (stop || !(beta > 0.0)) ? 0.0 : 1.0 / beta;
  } else if (lane == 0) {
    c.betaj[b] = 0.0;
    if (c.nbeta_f) c.nbeta_f[b] = make_float2(-0.0f, 0.0f);
  }
  if (lane == 0) c.sinv[b] = inv;
}

// q_next = w / beta into the next basis slot and xh = bf16(Delta^1/2 q_next)
// (beta, the breakdown test and 1/beta from k_beta_vec).  is_start: w
// holds b_tm; ||b|| from the partials here, beta0, and q_0 into slot 0.
__device__ __forceinline__ void normalize_chunk(const VecCtx &c, int j, int is_start, int chunk,
                                                int b) {
  const int v = c.vec0 + b;
  const bool real = b < c.nvec;
  bool live = real && is_start;
  __shared__ double sbeta, sinv;
  double inv = 0.0;
  if (!is_start) {
    inv = c.sinv[b];
    live = inv > 0.0;
  } else if (live) {
    // ||b||^2 from the per-chunk partials: one warp, fixed order, broadcast
    if (threadIdx.x < 32) {
      double s = 0.0;
      for (int ch = threadIdx.x; ch < c.nchunks; ch += 32) s += c.norm_a[(size_t)b * c.nchunks + ch];
      s = warp_sum(s);
      if (threadIdx.x == 0) {
        sbeta = sqrt(s);
        sinv = sbeta > 0.0 ? 1.0 / sbeta : 0.0;
      }
    }
    __syncthreads();
    const double beta = sbeta;
    if (chunk == 0 && threadIdx.x == 0) {
      c.beta0[v] = beta;
      c.k_eff[v] = beta > 0.0 ? c.k : 0;
      c.amax[b] = 0.0;
      c.betaj[b] = 0.0;
    }
    live = beta > 0.0;
    inv = live ? sinv : 0.0;
  } else if (chunk == 0 && threadIdx.x == 0) {
    c.betaj[b] = 0.0;
  }
  const int next = is_start ? 0 : j + 1;
  if (next >= c.nslots && c.reorth != LGW_REORTH_NONE) return;
  const size_t voff = (size_t)b * c.N;
  const int e0 = elem_base(chunk);
  if (c.pair) {
    // float-pair slots: the start reads the FP64 b of the start kernels,
    // a step the float-pair w of the axpy pass
    float *qh = pair_hi(slot_ptr(c, next), c) + voff, *ql = pair_lo(slot_ptr(c, next), c) + voff;
    const float *wh = pair_hi(c.w, c) + voff, *wl = pair_lo(c.w, c) + voff;
    const dfl si = df_from(inv);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * 64;
      if (e >= c.N) continue;
      dfl q0{0.f, 0.f}, q1{0.f, 0.f};
      if (live && is_start) {
        const double2 w2 = *reinterpret_cast<const double2 *>(c.w + voff + e);
        q0 = df_from(w2.x * inv);
        q1 = df_from(w2.y * inv);
      } else if (live) {
        const float2 x2 = *reinterpret_cast<const float2 *>(wh + e);
        const float2 y2 = *reinterpret_cast<const float2 *>(wl + e);
        q0 = df_mul({x2.x, y2.x}, si);
        q1 = df_mul({x2.y, y2.y}, si);
      }
      *reinterpret_cast<float2 *>(qh + e) = make_float2(q0.h, q1.h);
      *reinterpret_cast<float2 *>(ql + e) = make_float2(q0.l, q1.l);
      if (c.xh != nullptr) {
        __nv_bfloat162 x2;
        x2.x = __float2bfloat16_rn(c.dsqf[e] * q0.h);
        x2.y = __float2bfloat16_rn(c.dsqf[e + 1] * q1.h);
        *reinterpret_cast<__nv_bfloat162 *>(c.xh + kblk_bf16(b, e, c.Bs)) = x2;
      }
    }
    return;
  }
  double *qn = slot_ptr(c, next) + voff;
  const double *w = c.w + voff;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    if (e >= c.N) continue;
    double2 q2 = make_double2(0.0, 0.0);
    if (live) {
      q2 = *reinterpret_cast<const double2 *>(w + e);
      q2.x *= inv;
      q2.y *= inv;
    }
    *reinterpret_cast<double2 *>(qn + e) = q2;
    if (c.xh != nullptr) {
      // the BF16 operand from the FP32 image of q (FP64 multiplies and
      // FP64 -> BF16 conversions would load GB300's narrow FP64 pipe)
      __nv_bfloat162 x2;
      x2.x = __float2bfloat16_rn(c.dsqf[e] * __double2float_rn(q2.x));
      x2.y = __float2bfloat16_rn(c.dsqf[e + 1] * __double2float_rn(q2.y));
      *reinterpret_cast<__nv_bfloat162 *>(c.xh + kblk_bf16(b, e, c.Bs)) = x2;
    }
  }
}

__global__ void __launch_bounds__(VEC_THREADS) k_normalize(VecCtx c, int j, int is_start) {
  const int n = cpb_of(c), c0 = blockIdx.x * n, c1 = min(c.nchunks, c0 + n);
  for (int chunk = c0; chunk < c1; ++chunk) normalize_chunk(c, j, is_start, chunk, blockIdx.y);
}

// w = Delta^1/2 V for the rows of a given coupling block (V row stride ldv,
// n_valid real pair elements per row), zero elsewhere; ||w||^2 partials.
__global__ void __launch_bounds__(VEC_THREADS) k_start_from_v(VecCtx c, const double *V, int ldv,
                                                              int n_valid) {
  __shared__ double red[VEC_THREADS / 32];
  const int chunk = blockIdx.x, b = blockIdx.y;
  const size_t voff = (size_t)b * c.N;
  const int e0 = elem_base(chunk);
  double nrm = 0.0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    if (e >= c.N) continue;
    double x0 = 0.0, x1 = 0.0;
    if (b < c.nvec) {
      if (e < n_valid) x0 = c.dsq[e] * V[(size_t)b * ldv + e];
      if (e + 1 < n_valid) x1 = c.dsq[e + 1] * V[(size_t)b * ldv + e + 1];
    }
    c.w[voff + e] = x0;
    c.w[voff + e + 1] = x1;
    nrm = fma(x0, x0, fma(x1, x1, nrm));
  }
  nrm = block_sum(nrm, red);
  if (threadIdx.x == 0) c.norm_a[(size_t)b * c.nchunks + chunk] = nrm;
}

// w = Delta^1/2 * vf (float coupling vectors from the tensor cores) and
// ||w||^2 partials; padding vectors get zeros.
__global__ void __launch_bounds__(VEC_THREADS) k_start_from_vf(VecCtx c, const float *vf) {
  __shared__ double red[VEC_THREADS / 32];
  const int chunk = blockIdx.x, b = blockIdx.y;
  const size_t voff = (size_t)b * c.N;
  const int e0 = elem_base(chunk);
  double nrm = 0.0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    if (e >= c.N) continue;
    double x0 = 0.0, x1 = 0.0;
    if (b < c.nvec) {
      const float2 v2 = *reinterpret_cast<const float2 *>(vf + kblk_f32(b, e, c.Bs));
      x0 = c.dsq[e] * (double)v2.x;
      x1 = c.dsq[e + 1] * (double)v2.y;
    }
    *reinterpret_cast<double2 *>(c.w + voff + e) = make_double2(x0, x1);
    nrm = fma(x0, x0, fma(x1, x1, nrm));
  }
  nrm = block_sum(nrm, red);
  if (threadIdx.x == 0) c.norm_a[(size_t)b * c.nchunks + chunk] = nrm;
}

__global__ void __launch_bounds__(VEC_THREADS) k_norm_partials(VecCtx c, const double *x,
                                                               double *out) {
  __shared__ double red[VEC_THREADS / 32];
  const int chunk = blockIdx.x, b = blockIdx.y;
  const size_t voff = (size_t)b * c.N;
  const int e0 = elem_base(chunk);
  double nrm = 0.0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    if (e >= c.N || b >= c.nvec) continue;
    const double2 x2 = *reinterpret_cast<const double2 *>(x + voff + e);
    nrm = fma(x2.x, x2.x, fma(x2.y, x2.y, nrm));
  }
  nrm = block_sum(nrm, red);
  if (threadIdx.x == 0) out[(size_t)b * c.nchunks + chunk] = nrm;
}

// out = bf16(Delta^1/2 x) for x [Bs][N], written K-block-major (the GEMM1
// operand layout)
__global__ void k_scale_rows_to_bf16(const double *__restrict__ x, const double *__restrict__ dsq,
                                     int Bs, int N, __nv_bfloat16 *__restrict__ out) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t n = (size_t)Bs * N;
  if (i >= n) return;
  out[kblk_bf16((int)(i / N), (int)(i % N), Bs)] = __double2bfloat16(dsq[i % N] * x[i]);
}

// ---------------------------------------------------------------------------
// Band Lanczos (the band method for resolvent matrix elements cited after
// Eq. 14), one new vector per step with full reorthogonalisation.  Each
// group g (a summed orbital m) carries one recurrence; its start block is
// the p targets' vectors b_{t,m}.  The start vectors are orthonormalised one
// after the other, then step j applies C to basis vector q_j; both cases
// end in the same orthogonalise-and-append: w is projected out of all of
// the group's vectors twice (classical Gram-Schmidt in FP64), the
// coefficients of both passes are recorded (a column of R0 or of the banded
// T), and w / ||w|| becomes the next basis vector unless ||w|| fell below
// the breakdown scale.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool band_act(const BandCtx &bc, int b) {
  return b < bc.c.nvec && bc.act[b] != 0;
}

__global__ void k_band_init(BandCtx bc) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= bc.c.Bs) return;
  bc.nv[b] = 0;
  bc.act[b] = 0;
  bc.newrow[b] = -1;
  bc.inv[b] = 0.0;
  bc.scale[b] = 0.0;
  bc.tmax[b] = 0.0;
}

// mode 0 (a start vector): every real group; mode 1 (step j): the groups
// whose basis vector j exists.
__global__ void k_band_activate(BandCtx bc, int mode, int j) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= bc.c.Bs) return;
  bc.act[b] = (b < bc.c.nvec && (mode == 0 || j < bc.nv[b])) ? 1 : 0;
}

// The contraction operand of q_j: FP64 copy (FP64 contractions) or
// bf16(Delta^1/2 q_j); zeros for groups without vector j.
__global__ void __launch_bounds__(VEC_THREADS) k_band_operand(BandCtx bc, int j) {
  const VecCtx &c = bc.c;
  const int chunk = blockIdx.x, b = blockIdx.y;
  const bool act = band_act(bc, b);
  const size_t voff = (size_t)b * c.N;
  const double *q = slot_ptr(c, j) + voff;
  const int e0 = elem_base(chunk);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    if (e >= c.N) continue;
    const double2 q2 = act ? *reinterpret_cast<const double2 *>(q + e) : make_double2(0.0, 0.0);
    if (bc.xq != nullptr) *reinterpret_cast<double2 *>(bc.xq + voff + e) = q2;
    if (c.xh != nullptr) {
      __nv_bfloat162 x2;
      x2.x = __float2bfloat16_rn(c.dsqf[e] * __double2float_rn(q2.x));
      x2.y = __float2bfloat16_rn(c.dsqf[e + 1] * __double2float_rn(q2.y));
      *reinterpret_cast<__nv_bfloat162 *>(c.xh + kblk_bf16(b, e, c.Bs)) = x2;
    }
  }
}

// w = Delta^2 q_j + c_K Delta^1/2 L y   (Eq. 4; the contraction in FP32)
__global__ void __launch_bounds__(VEC_THREADS) k_band_assemble(BandCtx bc, int j,
                                                              const float *__restrict__ ucd) {
  const VecCtx &c = bc.c;
  const int chunk = blockIdx.x, b = blockIdx.y;
  if (!band_act(bc, b)) return;
  const size_t voff = (size_t)b * c.N;
  const double *q = slot_ptr(c, j) + voff;
  const int e0 = elem_base(chunk);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    if (e >= c.N) continue;
    const double2 q2 = *reinterpret_cast<const double2 *>(q + e);
    const float2 v2 = *reinterpret_cast<const float2 *>(ucd + kblk_f32(b, e, c.Bs));
    double2 w2;
    w2.x = fma(c.Delta2[e], q2.x, (double)v2.x);
    w2.y = fma(c.Delta2[e + 1], q2.y, (double)v2.y);
    *reinterpret_cast<double2 *>(c.w + voff + e) = w2;
  }
}

// Dots of w with the group's basis vectors; pass 1 also ||w||^2 (norm_a).
__global__ void __launch_bounds__(VEC_THREADS) k_band_dots(BandCtx bc, int pass) {
  __shared__ double red[VEC_THREADS / 32];
  __shared__ double sred[VEC_THREADS / 32][32];
  const VecCtx &c = bc.c;
  const int chunk = blockIdx.x, b = blockIdx.y;
  if (!band_act(bc, b)) return;
  const double *w = c.w + (size_t)b * c.N;
  const int e0 = elem_base(chunk);
  double wr[8];
  double nrm = 0.0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    double2 w2 = make_double2(0.0, 0.0);
    if (e < c.N) w2 = *reinterpret_cast<const double2 *>(w + e);
    wr[2 * u] = w2.x;
    wr[2 * u + 1] = w2.y;
    nrm = fma(w2.x, w2.x, fma(w2.y, w2.y, nrm));
  }
  if (pass == 1) {
    nrm = block_sum(nrm, red);
    if (threadIdx.x == 0) c.norm_a[(size_t)b * c.nchunks + chunk] = nrm;
  }
  dots_rows(c, bc.nv[b], b, chunk, wr, sred);
}

// h = sum over chunks (fixed order); hsum accumulates the two passes.
__global__ void k_band_reduce(BandCtx bc, int pass) {
  const VecCtx &c = bc.c;
  const int b = blockIdx.x;
  if (!band_act(bc, b)) return;
  const int n = bc.nv[b];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double *pp = c.dot_part + (size_t)b * c.nchunks * c.kmax1 + i;
    double s = 0.0;
    for (int ch = 0; ch < c.nchunks; ++ch) s += pp[(size_t)ch * c.kmax1];
    const size_t hi = (size_t)b * c.kmax1 + i;
    c.h[hi] = s;
    bc.hsum[hi] = pass == 1 ? s : bc.hsum[hi] + s;
  }
}

// w <- w - sum_i h_i q_i over the group's vectors; ||w||^2 partials
// (pass 1: norm_b, pass 2: norm_c).
__global__ void __launch_bounds__(VEC_THREADS) k_band_update(BandCtx bc, int pass) {
  extern __shared__ double hs[];
  __shared__ double red[VEC_THREADS / 32];
  const VecCtx &c = bc.c;
  const int chunk = blockIdx.x, b = blockIdx.y;
  if (!band_act(bc, b)) return;
  const int n = bc.nv[b];
  for (int i = threadIdx.x; i < n; i += VEC_THREADS) hs[i] = c.h[(size_t)b * c.kmax1 + i];
  __syncthreads();
  const size_t voff = (size_t)b * c.N;
  double *w = c.w + voff;
  const int e0 = elem_base(chunk);
  double2 wv[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    wv[u] = (e < c.N) ? *reinterpret_cast<const double2 *>(w + e) : make_double2(0.0, 0.0);
  }
  for (int i = 0; i < n; ++i) {
    const double hi = hs[i];
    const double *qrow = slot_ptr(c, i) + voff;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * 64;
      if (e < c.N) {
        const double2 q2 = *reinterpret_cast<const double2 *>(qrow + e);
        wv[u].x = fma(-hi, q2.x, wv[u].x);
        wv[u].y = fma(-hi, q2.y, wv[u].y);
      }
    }
  }
  double nrm = 0.0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    if (e < c.N) *reinterpret_cast<double2 *>(w + e) = wv[u];
    nrm = fma(wv[u].x, wv[u].x, fma(wv[u].y, wv[u].y, nrm));
  }
  nrm = block_sum(nrm, red);
  if (threadIdx.x == 0) (pass == 1 ? c.norm_b : c.norm_c)[(size_t)b * c.nchunks + chunk] = nrm;
}

// One warp per group: beta = ||w|| after both passes, the coefficient
// record and the breakdown test; sets the row to append (or -1).
__global__ void k_band_beta(BandCtx bc, int mode, int idx) {
  const VecCtx &c = bc.c;
  const int b = blockIdx.x, lane = threadIdx.x;
  if (!band_act(bc, b)) {
    if (lane == 0 && b < c.Bs) bc.newrow[b] = -1;
    return;
  }
  const int g = c.vec0 + b, p = bc.p, n = bc.nv[b];
  double s2 = 0.0, s0 = 0.0;
  for (int ch = lane; ch < c.nchunks; ch += 32) {
    s2 += c.norm_c[(size_t)b * c.nchunks + ch];
    s0 += c.norm_a[(size_t)b * c.nchunks + ch];
  }
  const double beta = sqrt(warp_sum(s2));
  const double norm0 = sqrt(warp_sum(s0));
  const double *hs = bc.hsum + (size_t)b * c.kmax1;
  bool append;
  if (mode == 0) {
    // start vector a = idx: b_a = sum_{i<n} hsum_i q_i + beta q_n
    const int a = idx;
    for (int i = lane; i < n; i += 32) bc.R0[((size_t)g * p + i) * p + a] = hs[i];
    const double sc = fmax(bc.scale[b], norm0);
    append = beta > c.tol * sc;
    if (lane == 0) {
      bc.scale[b] = sc;
      if (append) bc.R0[((size_t)g * p + n) * p + a] = beta;
    }
  } else {
    // step j = idx: T[i][j] = hsum_i for j <= i < n (d = i - j <= p - 1),
    // T[n][j] = beta for an appended vector (d = n - j <= p)
    const int j = idx;
    double tm = 0.0;
    for (int i = j + lane; i < n; i += 32) {
      bc.Tb[((size_t)g * c.k + j) * (p + 1) + (i - j)] = hs[i];
      tm = fmax(tm, fabs(hs[i]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tm = fmax(tm, __shfl_xor_sync(0xffffffffu, tm, o));
    const double tmax = fmax(bc.tmax[b], tm);
    append = n < c.k && beta > c.tol * tmax;
    if (lane == 0) {
      bc.tmax[b] = tmax;
      if (append) bc.Tb[((size_t)g * c.k + j) * (p + 1) + (n - j)] = beta;
    }
  }
  if (lane == 0) {
    bc.newrow[b] = append ? n : -1;
    bc.inv[b] = append ? 1.0 / beta : 0.0;
    if (append) bc.nv[b] = n + 1;
  }
}

// q_new = w / beta into the appended row.
__global__ void __launch_bounds__(VEC_THREADS) k_band_normalize(BandCtx bc) {
  const VecCtx &c = bc.c;
  const int chunk = blockIdx.x, b = blockIdx.y;
  if (b >= c.nvec) return;
  const int r = bc.newrow[b];
  if (r < 0) return;
  const double inv = bc.inv[b];
  const size_t voff = (size_t)b * c.N;
  double *qn = slot_ptr(c, r) + voff;
  const double *w = c.w + voff;
  const int e0 = elem_base(chunk);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    if (e >= c.N) continue;
    double2 q2 = *reinterpret_cast<const double2 *>(w + e);
    q2.x *= inv;
    q2.y *= inv;
    *reinterpret_cast<double2 *>(qn + e) = q2;
  }
}

__global__ void k_band_finish(BandCtx bc) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= bc.c.nvec) return;
  bc.keff[bc.c.vec0 + b] = min(bc.c.k, bc.nv[b]);
}

// T[i][j] of group g from the lower band (0 outside the band or past ke).
__device__ __forceinline__ double band_T(const double *Tg, int p, int ke, int i, int j) {
  const int lo = i < j ? i : j, d = i < j ? j - i : i - j;
  if (d > p || lo < 0 || i >= ke || j >= ke) return 0.0;
  return Tg[(size_t)lo * (p + 1) + d];
}

// One warp per (polarisation vector xi, group g): k_eff-step Lanczos on the
// group's ke x ke banded T from y = R0 x (Eq. 13 on the projected matrix),
// CGS2 against the stored vectors (scratch rows in global memory, lanes
// over the ke components).  y^T f(T) y then follows from this tridiagonal
// like any start vector's: Gauss rule, square-root map, fraction.
__global__ void k_band_small(const double *__restrict__ Tb, const double *__restrict__ R0,
                             const int *__restrict__ keff, int G, int k, int p,
                             const double *__restrict__ xs, int nx, double tol,
                             double *__restrict__ scratch, double *__restrict__ alpha,
                             double *__restrict__ beta, double *__restrict__ beta0,
                             int *__restrict__ keff_out) {
  const int warps = blockDim.x >> 5;
  const int wv = blockIdx.x * warps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (wv >= nx * G) return;
  const int xi = wv / G, g = wv % G;
  const int ke = keff[g];
  double *Q = scratch + (size_t)wv * (k + 2) * k;   // rows 0..ke-1: basis; row k: u
  double *u = Q + (size_t)k * k;
  double *al = alpha + (size_t)wv * k, *be = beta + (size_t)wv * k;
  for (int i = lane; i < k; i += 32) {
    al[i] = 0.0;
    be[i] = 0.0;
  }
  const double *Tg = Tb + (size_t)g * k * (p + 1);
  const double *Rg = R0 + (size_t)g * p * p;
  // y_i = sum_a R0[i][a] x_a (nonzero for i < p)
  double ss = 0.0;
  for (int i = lane; i < ke; i += 32) {
    double y = 0.0;
    if (i < p)
      for (int a = 0; a < p; ++a) y = fma(Rg[(size_t)i * p + a], xs[(size_t)xi * p + a], y);
    u[i] = y;
    ss = fma(y, y, ss);
  }
  const double b0 = sqrt(warp_sum(ss));
  if (lane == 0) beta0[wv] = b0;
  if (!(b0 > 0.0) || ke <= 0) {
    if (lane == 0) keff_out[wv] = 0;
    return;
  }
  int kk = ke;
  double bprev = 0.0, amax = 0.0;
  double inv = 1.0 / b0;
  for (int j = 0; j < ke; ++j) {
    double *q = Q + (size_t)j * k;
    __syncwarp();
    for (int i = lane; i < ke; i += 32) q[i] = u[i] * inv;
    __syncwarp();
    // u = T q - beta_j q_{j-1}; alpha_j = q . u; u -= alpha_j q
    double aj = 0.0;
    for (int i = lane; i < ke; i += 32) {
      double s = 0.0;
      for (int d = -p; d <= p; ++d) {
        const int c2 = i + d;
        if (c2 >= 0 && c2 < ke) s = fma(band_T(Tg, p, ke, i, c2), q[c2], s);
      }
      if (j > 0) s = fma(-bprev, Q[(size_t)(j - 1) * k + i], s);
      u[i] = s;
      aj = fma(q[i], s, aj);
    }
    aj = warp_sum(aj);
    __syncwarp();
    for (int i = lane; i < ke; i += 32) u[i] = fma(-aj, q[i], u[i]);
    // full reorthogonalisation, twice
    for (int pass = 0; pass < 2; ++pass) {
      for (int r = 0; r <= j; ++r) {
        const double *qr = Q + (size_t)r * k;
        __syncwarp();
        double d = 0.0;
        for (int i = lane; i < ke; i += 32) d = fma(qr[i], u[i], d);
        d = warp_sum(d);
        __syncwarp();
        for (int i = lane; i < ke; i += 32) u[i] = fma(-d, qr[i], u[i]);
      }
    }
    __syncwarp();
    double nn = 0.0;
    for (int i = lane; i < ke; i += 32) nn = fma(u[i], u[i], nn);
    const double bj = sqrt(warp_sum(nn));
    amax = fmax(amax, fabs(aj));
    if (lane == 0) {
      al[j] = aj;
      be[j] = bj;
    }
    if (!(bj > tol * amax) || j + 1 == ke) {
      kk = j + 1;
      break;
    }
    bprev = bj;
    inv = 1.0 / bj;
  }
  if (lane == 0) keff_out[wv] = kk;
}

__global__ void k_band_combine(const double *__restrict__ sig, int p, int F,
                               double *__restrict__ out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const int ab = blockIdx.y;
  if (f >= F) return;
  const int a = ab / p, b = ab % p;
  double re, im;
  if (a == b) {
    re = sig[((size_t)a * F + f) * 2];
    im = sig[((size_t)a * F + f) * 2 + 1];
  } else {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    // pair index of (lo, hi) in the order (0,1), (0,2), ..., (1,2), ...
    const int q = lo * p - lo * (lo + 1) / 2 + (hi - lo - 1);
    const size_t xp = (size_t)(p + 2 * q), xm = xp + 1;
    re = 0.25 * (sig[(xp * F + f) * 2] - sig[(xm * F + f) * 2]);
    im = 0.25 * (sig[(xp * F + f) * 2 + 1] - sig[(xm * F + f) * 2 + 1]);
  }
  out[((size_t)ab * F + f) * 2] = re;
  out[((size_t)ab * F + f) * 2 + 1] = im;
}

// ---------------------------------------------------------------------------
static dim3 vec_grid(const VecCtx &c) { return dim3(c.nchunks, c.Bs); }

void launch_band_init(const BandCtx &bc, cudaStream_t st) {
  k_band_init<<<(bc.c.Bs + 255) / 256, 256, 0, st>>>(bc);
}
void launch_band_activate(const BandCtx &bc, int mode, int j, cudaStream_t st) {
  k_band_activate<<<(bc.c.Bs + 255) / 256, 256, 0, st>>>(bc, mode, j);
}
void launch_band_operand(const BandCtx &bc, int j, cudaStream_t st) {
  k_band_operand<<<vec_grid(bc.c), VEC_THREADS, 0, st>>>(bc, j);
}
void launch_band_assemble(const BandCtx &bc, int j, const float *ucd, cudaStream_t st) {
  k_band_assemble<<<vec_grid(bc.c), VEC_THREADS, 0, st>>>(bc, j, ucd);
}
int launch_band_append(const BandCtx &bc, int mode, int idx, cudaStream_t st) {
  const size_t sh = (size_t)bc.c.kmax1 * sizeof(double);
  for (int pass = 1; pass <= 2; ++pass) {
    k_band_dots<<<vec_grid(bc.c), VEC_THREADS, 0, st>>>(bc, pass);
    k_band_reduce<<<bc.c.Bs, 256, 0, st>>>(bc, pass);
    k_band_update<<<vec_grid(bc.c), VEC_THREADS, sh, st>>>(bc, pass);
  }
  k_band_beta<<<bc.c.Bs, 32, 0, st>>>(bc, mode, idx);
  k_band_normalize<<<vec_grid(bc.c), VEC_THREADS, 0, st>>>(bc);
  return 8;
}
void launch_band_finish(const BandCtx &bc, cudaStream_t st) {
  k_band_finish<<<(bc.c.Bs + 255) / 256, 256, 0, st>>>(bc);
}
void launch_band_small(const double *Tb, const double *R0, const int *keff, int G, int k, int p,
                       const double *xs, int nx, double tol, double *scratch, double *alpha,
                       double *beta, double *beta0, int *keff_out, cudaStream_t st) {
  const int warps = 4;
  const int n = nx * G;
  k_band_small<<<(n + warps - 1) / warps, 32 * warps, 0, st>>>(
      Tb, R0, keff, G, k, p, xs, nx, tol, scratch, alpha, beta, beta0, keff_out);
}
void launch_band_combine(const double *sig, int p, int F, double *out, cudaStream_t st) {
  dim3 grid((F + 127) / 128, p * p);
  k_band_combine<<<grid, 128, 0, st>>>(sig, p, F, out);
}

void launch_start_from_v(const VecCtx &c, const double *V, int ldv, int n_valid, cudaStream_t st) {
  k_start_from_v<<<vec_grid(c), VEC_THREADS, 0, st>>>(c, V, ldv, n_valid);
}
void launch_start_from_vf(const VecCtx &c, const float *vf, cudaStream_t st) {
  k_start_from_vf<<<vec_grid(c), VEC_THREADS, 0, st>>>(c, vf);
}
void launch_norm_partials(const VecCtx &c, const double *x, double *out, cudaStream_t st) {
  k_norm_partials<<<vec_grid(c), VEC_THREADS, 0, st>>>(c, x, out);
}
// grid of the kernels that take c.cpb chunks per block
static dim3 vec_grid_cpb(const VecCtx &c) {
  const int n = c.cpb > 1 ? c.cpb : 1;
  return dim3((c.nchunks + n - 1) / n, c.Bs);
}
void launch_normalize(const VecCtx &c, int j, int is_start, const double *, cudaStream_t st) {
  k_normalize<<<vec_grid_cpb(c), VEC_THREADS, 0, st>>>(c, j, is_start);
}
void launch_assemble_w(const VecCtx &c, int j, const float *ucd, cudaStream_t st) {
  k_assemble_w<<<vec_grid_cpb(c), VEC_THREADS, 0, st>>>(c, j, ucd);
}
void launch_alpha_reduce(const VecCtx &c, int j, cudaStream_t st) {
  k_alpha_reduce<<<c.Bs, 32, 0, st>>>(c, j);
}
void launch_alpha_axpy(const VecCtx &c, int j, cudaStream_t st) {
  if (c.reorth != LGW_REORTH_NONE)
    k_alpha_axpy<true><<<vec_grid_cpb(c), VEC_THREADS, 0, st>>>(c, j);
  else
    k_alpha_axpy<false><<<vec_grid_cpb(c), VEC_THREADS, 0, st>>>(c, j);
}
void launch_beta_vec(const VecCtx &c, int j, cudaStream_t st) {
  k_beta_vec<<<c.Bs, 32, 0, st>>>(c, j);
}
void launch_reduce_dots(const VecCtx &c, int j, int pass, cudaStream_t st) {
  k_reduce_dots<<<c.Bs, 256, 0, st>>>(c, j, pass);
}
void launch_update(const VecCtx &c, int j, int pass, cudaStream_t st) {
  size_t sh = (size_t)c.kmax1 * sizeof(double);
  k_update<<<vec_grid(c), VEC_THREADS, sh, st>>>(c, j, pass);
}
void launch_dots(const VecCtx &c, int j, int, cudaStream_t st) {
  k_dots<<<vec_grid(c), VEC_THREADS, 0, st>>>(c, j);
}
void launch_second_pass_decide_j(const VecCtx &c, int j, cudaStream_t st) {
  k_second_pass_decide<<<(c.Bs + 255) / 256, 256, 0, st>>>(c, j);
}
void launch_scale_rows_to_bf16(const double *x, const double *dsq, int Bs, int N,
                               __nv_bfloat16 *out, cudaStream_t st) {
  size_t n = (size_t)Bs * N;
  k_scale_rows_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, dsq, Bs, N, out);
}

}  // namespace lgw
