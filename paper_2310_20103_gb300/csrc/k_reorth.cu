// Full reorthogonalisation against a split-precision Krylov basis.
//
// GB300 executes FP64 at ~1/58 of its FP32 rate (1.2 vs 70 TFLOP/s), so a
// Gram-Schmidt pass with one DFMA per 8-byte basis element stalls on the FP64
// pipe well below HBM bandwidth.  Here every basis vector q_i is stored as a
// pair of floats (q_hi = fl32(q), q_lo = fl32(q - q_hi); q_hi + q_lo carries
// 48 significant bits) and the recurrence keeps exact FP64 copies of
// q_{j-1}, q_j, q_{j+1} in a three-slot ring.
//
//  dots   h_i = q_i . w in double-float arithmetic on the FP32 pipe: the
//         product q_hi w_hi is split exactly with an FMA, the cross terms are
//         added in FP32, and the running sum is a (hi, lo) pair updated by
//         Knuth's TwoSum (non-contracted intrinsics).  Relative error of a
//         partial ~2^-48 of sum |q_i,e w_e|, comparable to FP64 summation.
//  alpha  alpha_j = q_j . w from the contraction epilogue's partials, and
//         w <- w - alpha_j q_j in FP64 (exact q_j from the ring) BEFORE the
//         projections, as in the three-term recurrence of Eq. 13.  Projecting
//         alpha_j q_j out inside classical Gram-Schmidt instead would leave
//         residues ~ ||Q^T Q - I|| alpha_j / beta_{j+1} that grow every step.
//  update w <- w - sum_i h_i q_i.  After the alpha subtraction every h_i is
//         O(eps ||w||) (or O(u_bf16 ||w||) from the slight asymmetry of the
//         BF16 operator), so the sum is formed in FP32 from q_hi alone (4
//         bytes per element); its rounding is far below the FP64 resolution
//         of w.  The second pass (where taken) is identical.
//  norm   ||w - Q h||^2 = ||w||^2 - ||h||^2 gives beta_{j+1} before the
//         update, so the update pass that finishes a vector also writes
//         q_{j+1} = (w - Q h) / beta_{j+1} in every form the next step reads,
//         and w is not stored and re-read for a separate normalisation.
//
// Block layout as in the FP64 kernels: one block per (chunk of VEC_CHUNK
// elements, vector), eight elements per thread.
#include "lgw_internal.cuh"

namespace lgw {

__device__ __forceinline__ int elem_base_s(int chunk) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  return chunk * VEC_CHUNK + wid * 256 + 2 * lane;
}

__device__ __forceinline__ bool live_s(const VecCtx &c, int b, int j) {
  return b < c.nvec && c.k_eff[c.vec0 + b] > j;
}

// (s_hi, s_lo) += p exactly representable part via TwoSum; never contracted.
__device__ __forceinline__ void two_sum_acc(float &s_hi, float &s_lo, float p) {
  const float s = __fadd_rn(s_hi, p);
  const float bb = __fsub_rn(s, s_hi);
  const float err = __fadd_rn(__fsub_rn(s_hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  s_hi = s;
  s_lo = __fadd_rn(s_lo, err);
}

// Double-float sum of two (hi, lo) pairs.
__device__ __forceinline__ void df_add(float &ah, float &al, float bh, float bl) {
  const float s = __fadd_rn(ah, bh);
  const float bb = __fsub_rn(s, ah);
  const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  ah = s;
  al = __fadd_rn(__fadd_rn(al, bl), err);
}

__device__ __forceinline__ const float *bhi_row(const VecCtx &c, int i, int b) {
  return c.bhi + ((size_t)i * c.Bs + b) * c.N;
}
__device__ __forceinline__ const float *blo_row(const VecCtx &c, int i, int b) {
  return c.blo + ((size_t)i * c.Bs + b) * c.N;
}

// One lane's share of a row . w over a VEC_CHUNK chunk in double-float:
// four quarters of 512 elements, each lane a float4 of hi and of lo per 128
// elements (4 + 4 independent 128-bit loads per quarter).
template <bool LO>
__device__ __forceinline__ void dot_row_df(const float *__restrict__ qh,
                                           const float *__restrict__ ql, const float *swh,
                                           const float *swl, int lane, int nvalid, float &sh,
                                           float &sl) {
#pragma unroll
  for (int qt = 0; qt < 4; ++qt) {
    float4 hv[4], lv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int off = qt * 512 + 128 * t + 4 * lane;
      if (off < nvalid) {
        hv[t] = __ldg(reinterpret_cast<const float4 *>(qh + off));
        lv[t] = LO ? __ldg(reinterpret_cast<const float4 *>(ql + off))
                   : make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        hv[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        lv[t] = hv[t];
      }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int off = qt * 512 + 128 * t + 4 * lane;
      const float4 a = *reinterpret_cast<const float4 *>(swh + off);
      const float4 al = *reinterpret_cast<const float4 *>(swl + off);
      const float qa[4] = {hv[t].x, hv[t].y, hv[t].z, hv[t].w};
      const float qb[4] = {lv[t].x, lv[t].y, lv[t].z, lv[t].w};
      const float wa[4] = {a.x, a.y, a.z, a.w};
      const float wb[4] = {al.x, al.y, al.z, al.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float pr = __fmul_rn(qa[q], wa[q]);
        float err = __fmaf_rn(qa[q], wa[q], -pr);
        err = __fmaf_rn(qa[q], wb[q], err);
        err = __fmaf_rn(qb[q], wa[q], err);
        two_sum_acc(sh, sl, pr);
        sl = __fadd_rn(sl, err);
      }
    }
  }
}

// Dot products of w with basis rows 0..j.  Pass 1 first finishes alpha_j,
// applies w <- w - alpha_j q_j and writes ||w||^2 partials (norm_a).
//
// The block's chunk of w is split once into (hi, lo) floats in shared memory;
// then each warp takes whole rows (i = warp, warp + 8, ...) over the chunk:
// every lane streams 8 independent 128-bit loads per quarter row, accumulates
// its 64 products in double-float, and one 5-step butterfly gives the row's
// partial.  No block barrier inside the row loop.
template <int PASS>
__global__ void __launch_bounds__(VEC_THREADS, 2) k_dots_split(VecCtx c, int j) {
  __shared__ __align__(16) float swh[VEC_CHUNK];
  __shared__ __align__(16) float swl[VEC_CHUNK];
  __shared__ double red[VEC_THREADS / 32];
  const int chunk = blockIdx.x, b = blockIdx.y;
  if (!live_s(c, b, j)) return;
  if (PASS == 2 && !c.flag2[b]) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double alpha = 0.0;
  if (PASS == 1) {
    double s = 0.0;
    if (c.ucd != nullptr) {
      // estimate alpha_j = sum Delta^2 q_j^2 + c_K y . bf16(y)  (y = L^T Delta^1/2 q_j,
      // so q_j . c_K Delta^1/2 L y_hat = c_K y . y_hat); beta_j q_j . q_{j-1} ~ 0.
      for (int t = threadIdx.x; t < c.nchunks; t += VEC_THREADS)
        s += (double)c.dq2_part[(size_t)b * c.nchunks + t];
      for (int t = threadIdx.x; t < c.n_yb; t += VEC_THREADS)
        s += c.kf * (double)c.yy_part[(size_t)b * c.n_yb + t];
    } else {
      for (int t = threadIdx.x; t < c.n_mt; t += VEC_THREADS)
        s += c.alpha_part[(size_t)t * c.Bs + b];
    }
    alpha = block_sum(s, red);
    // alpha used for the subtraction; k_reduce_dots_split adds the residual
    // projection h_j so the recorded alpha_j is the FP64 Rayleigh quotient
    if (chunk == 0 && threadIdx.x == 0) c.alpha[(size_t)(c.vec0 + b) * c.k + j] = alpha;
  }
  double *w = c.w + (size_t)b * c.N;
  const double *qj = slot_ptr(c, j) + (size_t)b * c.N;
  const double *qp = (j >= 1) ? slot_ptr(c, j - 1) + (size_t)b * c.N : nullptr;
  const float *ucd = c.ucd;
  const double bj = c.betaj[b];
  const int cbase = chunk * VEC_CHUNK;
  const int e0 = elem_base_s(chunk);
  double nrm = 0.0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    double2 w2 = make_double2(0.0, 0.0);
    if (e < c.N) {
      if (PASS == 1) {
        const double2 q2 = *reinterpret_cast<const double2 *>(qj + e);
        if (ucd != nullptr) {
          // w = Delta^2 q_j + c_K Delta^1/2 (L y) - beta_j q_{j-1}   (Eq. 4, 13)
          const float2 u2 = *reinterpret_cast<const float2 *>(ucd + kblk_f32(b, e, c.Bs));
          w2.x = fma(c.Delta2[e], q2.x, (double)u2.x);
          w2.y = fma(c.Delta2[e + 1], q2.y, (double)u2.y);
          if (qp != nullptr) {
            const double2 p2 = *reinterpret_cast<const double2 *>(qp + e);
            w2.x = fma(-bj, p2.x, w2.x);
            w2.y = fma(-bj, p2.y, w2.y);
          }
        } else {
          w2 = *reinterpret_cast<const double2 *>(w + e);
        }
        w2.x = fma(-alpha, q2.x, w2.x);
        w2.y = fma(-alpha, q2.y, w2.y);
        *reinterpret_cast<double2 *>(w + e) = w2;
      } else {
        w2 = *reinterpret_cast<const double2 *>(w + e);
      }
    }
    nrm = fma(w2.x, w2.x, fma(w2.y, w2.y, nrm));
    const float hx = __double2float_rn(w2.x), hy = __double2float_rn(w2.y);
    const int le = e - cbase;
    swh[le] = hx;
    swh[le + 1] = hy;
    swl[le] = __double2float_rn(w2.x - (double)hx);
    swl[le + 1] = __double2float_rn(w2.y - (double)hy);
  }
  if (PASS == 1) {
    nrm = block_sum(nrm, red);   // contains a __syncthreads
    if (threadIdx.x == 0) c.norm_a[(size_t)b * c.nchunks + chunk] = nrm;
  } else {
    __syncthreads();
  }
  const int nvalid = min(VEC_CHUNK, c.N - cbase);   // multiple of 128
  double *dp = c.dot_part + ((size_t)b * c.nchunks + chunk) * c.kmax1;
  for (int i = wid; i <= j; i += VEC_THREADS / 32) {
    const float *qh = bhi_row(c, i, b) + cbase;
    float sh = 0.f, sl = 0.f;
    if (c.blo != nullptr)
      dot_row_df<true>(qh, blo_row(c, i, b) + cbase, swh, swl, lane, nvalid, sh, sl);
    else
      dot_row_df<false>(qh, nullptr, swh, swl, lane, nvalid, sh, sl);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const float rh = __shfl_xor_sync(0xffffffffu, sh, o);
      const float rl = __shfl_xor_sync(0xffffffffu, sl, o);
      df_add(sh, sl, rh, rl);
    }
    if (lane == 0) dp[i] = (double)sh + (double)sl;
  }
}

// h[b][i] = sum over chunks (fixed order), then the norm of the projected
// vector without reading it back: with Q orthonormal,
//   ||w - Q h||^2 = ||w||^2 - ||h||^2,
// where the error of the right side (dot-product rounding, ~2^-48 ||w||
// per h_i, and the departure of Q^T Q from I, met only through the small
// h) is far below the FP64 resolution of ||w||^2 whenever no second pass
// is due.  Pass 1 decides the second pass from it (CGS2: always; CGS1K:
// when the first pass removes more than half of ||w||^2, the 1/sqrt(2)
// criterion); every vector that takes no second pass gets beta_{j+1}, the
// breakdown test and 1/beta here (pass 2: the others, from the measured
// ||w'||^2 of pass 1), and its update kernel writes q_{j+1} directly.
// Not-live vectors get flag2 = 0 and 1/beta = 0, so the update writes
// zeros into their next slot.
__global__ void __launch_bounds__(256) k_reduce_dots_split(VecCtx c, int j, int pass) {
  __shared__ double red[256 / 32];
  const int b = blockIdx.x;
  const int v = c.vec0 + b;
  if (!live_s(c, b, j)) {
    if (pass == 1 && threadIdx.x == 0) {
      c.flag2[b] = 0;
      c.sinv[b] = 0.0;
      c.betaj[b] = 0.0;
    }
    return;
  }
  if (pass == 2 && !c.flag2[b]) return;
  double hh = 0.0;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const double *p = c.dot_part + (size_t)b * c.nchunks * c.kmax1 + i;
    double s = 0.0;
    for (int ch = 0; ch < c.nchunks; ++ch) s += p[(size_t)ch * c.kmax1];
    c.h[(size_t)b * c.kmax1 + i] = s;
    hh = fma(s, s, hh);
    if (pass == 1 && i == j) {
      const size_t ai = (size_t)v * c.k + j;
      const double a = c.alpha[ai] + s;
      c.alpha[ai] = a;
      c.amax[b] = fmax(c.amax[b], fabs(a));
    }
  }
  const double *np = (pass == 1 ? c.norm_a : c.norm_b) + (size_t)b * c.nchunks;
  double nw = 0.0;
  for (int ch = threadIdx.x; ch < c.nchunks; ch += blockDim.x) nw += np[ch];
  hh = block_sum(hh, red);   // the barriers also publish amax[b]
  nw = block_sum(nw, red);
  if (threadIdx.x != 0) return;
  const double rest = nw - hh;   // ||w - Q h||^2
  int f = 0;
  if (pass == 1) {
    f = c.reorth == LGW_REORTH_CGS2 ? 1 : (rest < 0.5 * nw);
    c.flag2[b] = f;
    if (f && c.reorth != LGW_REORTH_CGS2) atomicAdd(c.n_second, 1);
  }
  if (f) return;
  const double beta = sqrt(fmax(rest, 0.0));
  const bool stop = !(beta > c.tol * c.amax[b]);
  c.beta[(size_t)v * c.k + j] = beta;
  c.betaj[b] = beta;
  if (stop) c.k_eff[v] = j + 1;
  c.sinv[b] = (stop || !(beta > 0.0)) ? 0.0 : 1.0 / beta;
}

// w <- w - Q h with every coefficient small: FP32 products and sum from q_hi.
// A vector whose beta_{j+1} is already known (no second pass after this
// one) is normalised in the same pass: q_{j+1} = (w - Q h) / beta_{j+1}
// into the FP64 ring, the split basis slot and the bf16 contraction
// operand, with the per-chunk partials of sum Delta^2 q_{j+1}^2; w itself is
// not written back.  A vector due for a second pass stores w and its norm
// partials instead.  Not-live vectors (padding, stopped) get zeros in their
// next slot.
template <int PASS>
__global__ void __launch_bounds__(VEC_THREADS) k_update_split(VecCtx c, int j) {
  extern __shared__ float hsf[];
  __shared__ double red[VEC_THREADS / 32];
  __shared__ float sdq[VEC_THREADS / 32];
  const int chunk = blockIdx.x, b = blockIdx.y;
  const bool live = live_s(c, b, j);
  const bool f2 = live && c.flag2[b];
  if (PASS == 2 && !f2) return;
  const bool fin = PASS == 2 || !f2;            // this launch writes q_{j+1}
  const double inv = (fin && live) ? c.sinv[b] : 0.0;
  const bool work = fin ? inv > 0.0 : true;     // w - Q h is needed
  const size_t voff = (size_t)b * c.N;
  double *w = c.w + voff;
  const int e0 = elem_base_s(chunk);
  float r[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) r[t] = 0.f;
  if (work) {
    const double *hb = c.h + (size_t)b * c.kmax1;
    const int nrows = j + 1;
    for (int i = threadIdx.x; i < nrows; i += VEC_THREADS) hsf[i] = (float)hb[i];
    __syncthreads();
    // four rows per trip keep sixteen independent loads in flight per thread
#pragma unroll 4
    for (int i = 0; i < nrows; ++i) {
      const float hf = hsf[i];
      const float *qh = bhi_row(c, i, b);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * 64;
        if (e < c.N) {
          const float2 q2 = *reinterpret_cast<const float2 *>(qh + e);
          r[2 * u] = fmaf(hf, q2.x, r[2 * u]);
          r[2 * u + 1] = fmaf(hf, q2.y, r[2 * u + 1]);
        }
      }
    }
  }
  if (!fin) {
    double nrm = 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * 64;
      if (e >= c.N) continue;
      double2 w2 = *reinterpret_cast<const double2 *>(w + e);
      w2.x -= (double)r[2 * u];
      w2.y -= (double)r[2 * u + 1];
      *reinterpret_cast<double2 *>(w + e) = w2;
      nrm = fma(w2.x, w2.x, fma(w2.y, w2.y, nrm));
    }
    nrm = block_sum(nrm, red);
    if (threadIdx.x == 0) c.norm_b[(size_t)b * c.nchunks + chunk] = nrm;
    return;
  }
  const int next = j + 1;
  double *qn = slot_ptr(c, next) + voff;
  float *hn = c.bhi + ((size_t)next * c.Bs + b) * c.N;
  float *ln = c.blo ? c.blo + ((size_t)next * c.Bs + b) * c.N : nullptr;
  float dq = 0.0f;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    if (e >= c.N) continue;
    double2 q2 = make_double2(0.0, 0.0);
    if (work) {
      q2 = *reinterpret_cast<const double2 *>(w + e);
      q2.x = (q2.x - (double)r[2 * u]) * inv;
      q2.y = (q2.y - (double)r[2 * u + 1]) * inv;
    }
    *reinterpret_cast<double2 *>(qn + e) = q2;
    const float hx = __double2float_rn(q2.x), hy = __double2float_rn(q2.y);
    dq = fmaf(c.d2f[e] * hx, hx, fmaf(c.d2f[e + 1] * hy, hy, dq));
    *reinterpret_cast<float2 *>(hn + e) = make_float2(hx, hy);
    if (ln != nullptr)
      *reinterpret_cast<float2 *>(ln + e) = make_float2(__double2float_rn(q2.x - (double)hx),
                                                        __double2float_rn(q2.y - (double)hy));
    if (c.xh != nullptr) {
      __nv_bfloat162 x2;
      x2.x = __float2bfloat16_rn(c.dsqf[e] * hx);
      x2.y = __float2bfloat16_rn(c.dsqf[e + 1] * hy);
      *reinterpret_cast<__nv_bfloat162 *>(c.xh + kblk_bf16(b, e, c.Bs)) = x2;
    }
  }
  if (c.dq2_part != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dq += __shfl_xor_sync(0xffffffffu, dq, o);
    if ((threadIdx.x & 31) == 0) sdq[threadIdx.x >> 5] = dq;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.0f;
      for (int w8 = 0; w8 < VEC_THREADS / 32; ++w8) t += sdq[w8];
      c.dq2_part[(size_t)b * c.nchunks + chunk] = t;
    }
  }
}

// q_0 = b / ||b|| (b = Delta^1/2 L M in w, its norm partials in norm_a)
// into ring slot 0, the split basis slot 0 and the bf16 contraction
// operand; beta0, k_eff and the per-vector state of the recurrence.
__global__ void __launch_bounds__(VEC_THREADS) k_start_split(VecCtx c) {
  const int chunk = blockIdx.x, b = blockIdx.y;
  const int v = c.vec0 + b;
  __shared__ double sbeta, sinv;
  __shared__ float sdq[VEC_THREADS / 32];
  bool live = b < c.nvec;
  double inv = 0.0;
  if (live) {
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
      c.sinv[b] = beta > 0.0 ? 1.0 : 0.0;   // q_0 is carried normalised
    }
    live = beta > 0.0;
    inv = sinv;
  } else if (chunk == 0 && threadIdx.x == 0) {
    c.betaj[b] = 0.0;
    c.sinv[b] = 0.0;
  }
  const size_t voff = (size_t)b * c.N;
  double *qn = slot_ptr(c, 0) + voff;
  float *hn = c.bhi + (size_t)b * c.N;
  float *ln = c.blo ? c.blo + (size_t)b * c.N : nullptr;
  const double *w = c.w + voff;
  const int e0 = elem_base_s(chunk);
  float dq = 0.0f;
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
    const float hx = __double2float_rn(q2.x), hy = __double2float_rn(q2.y);
    dq = fmaf(c.d2f[e] * hx, hx, fmaf(c.d2f[e + 1] * hy, hy, dq));
    *reinterpret_cast<float2 *>(hn + e) = make_float2(hx, hy);
    if (ln != nullptr)
      *reinterpret_cast<float2 *>(ln + e) = make_float2(__double2float_rn(q2.x - (double)hx),
                                                        __double2float_rn(q2.y - (double)hy));
    if (c.xh != nullptr) {
      __nv_bfloat162 x2;
      x2.x = __float2bfloat16_rn(c.dsqf[e] * hx);
      x2.y = __float2bfloat16_rn(c.dsqf[e + 1] * hy);
      *reinterpret_cast<__nv_bfloat162 *>(c.xh + kblk_bf16(b, e, c.Bs)) = x2;
    }
  }
  if (c.dq2_part != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dq += __shfl_xor_sync(0xffffffffu, dq, o);
    if ((threadIdx.x & 31) == 0) sdq[threadIdx.x >> 5] = dq;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.0f;
      for (int w8 = 0; w8 < VEC_THREADS / 32; ++w8) t += sdq[w8];
      c.dq2_part[(size_t)b * c.nchunks + chunk] = t;
    }
  }
}

// ===========================================================================
// Delayed classical Gram-Schmidt (LGW_REORTH_DCGS): one pass over the
// stored basis per step.
//
// Step j receives the carried vector w_{j-1} (c.wv, not normalised),
// 1/beta_j (c.sinv) and the projection coefficients h = Q_{j-1}^T w_{j-1}
// of the previous step (c.h), whose update has not been applied yet.  The
// contractions of this step already ran on q~_j = w_{j-1} / beta_j.  The
// basis vector is q_j = q~_j - Q_{j-1} h / beta_j.  Since C is linear,
//   C q_j = C q~_j - Q_{j-1} T_{j-1} h / beta_j - h_{j-1} q_j + O(eps |h|),
// i.e. C q~_j differs from C q_j by a vector of span(Q_j).  So the step
// forms, per element (Eq. 13 with the estimate alpha~_j),
//   v = C q~_j - alpha~_j q~_j - beta_j q_{j-1},
// and the projection of v on Q_j removes everything the delay changed:
// v - Q_j Q_j^T v equals the exactly recurred, fully reorthogonalised w_j,
// and the q_j coefficient h'_j = q_j . v = alpha_j - alpha~_j + h_{j-1}
// gives the FP64 Rayleigh quotient alpha_j = alpha~_j + h'_j - h_{j-1}.
// The span(Q_{j-1}) part of v is known before the sweep: with c = h/beta_j,
//   Q_{j-1}^T v = g + (rounding),   g = (T_{j-1} - alpha~_j) c,
// T_{j-1} being the tridiagonal recorded so far.  If it stayed in the
// carried vector, the next step's contraction would map it through T again
// and the carried components would grow by ||T - alpha~||/beta every step
// (the delay never cleans the vector).  So the sweep also subtracts Q_{j-1} g:
// in one pass over the rows q_i (i < j) each element accumulates
//   d_i  += q_i . v          (double-float, as k_dots_split)
//   corr += c_i q_i          (FP32 from q_hi: every c_i is small)
//   cv   += g_i q_i          (FP32 from q_hi: every g_i is small)
// and then writes q_j = q~_j - corr into row j of the basis, the next
// carried vector w_j = v - cv, the bf16 operand Delta^1/2 w_j (the
// reduction after GEMM1 scales the contraction by 1/beta_{j+1}) and the
// partials of q_j . w_j, ||w_j||^2 and sum Delta^2 w_j^2.  The reduction
// takes Q_{j-1}^T w_j = d - g (Q orthonormal).  Bytes per element and step:
// 8 per stored row (hi + lo) + 30, against 12 per row + 54 for the two
// passes of k_dots_split and k_update_split.
//
// Thread layout: one block per (2048-element chunk, vector); each thread
// owns elements e = chunk*2048 + warp*256 + 4*lane + 128*u + {0..3},
// u = 0, 1, for all rows, so the correction needs no cross-thread sum.
// Each row's dot partial is reduced by a double-float butterfly per warp
// and across the eight warps through shared memory, 32 rows at a time.
// ===========================================================================

// ---------------------------------------------------------------------------
// Row staging for the sweep: every thread copies the 8 elements of each row
// that it consumes (hi and lo, four 16-byte pieces) into its own slots of a
// shared-memory ring with cp.async, SW_SLOTS rows ahead, and reads them back
// two rows at a time.  No thread reads another's slots, so the ring needs
// no barrier; memory parallelism no longer competes with registers
// (4 rows x 64 bytes in flight per thread while 2 rows are computed).
// ---------------------------------------------------------------------------
constexpr int SW_SLOTS = 6;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                   (unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
// the same with immediate byte offsets on both addresses
template <int SOFF, int GOFF>
__device__ __forceinline__ void cp_async16_at(uint32_t saddr, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0+%2], [%1+%3], 16;\n" ::"r"(saddr), "l"(gmem),
               "n"(SOFF), "n"(GOFF)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Staging bytes per block.
template <bool LO>
__host__ __device__ constexpr size_t sweep_stage_bytes() {
  return (size_t)SW_SLOTS * (LO ? 4 : 2) * VEC_THREADS * sizeof(float4);
}

// Packed FP32 pairs: one instruction rounds each of the two lanes to nearest,
// exactly as the scalar __fadd_rn / __fmul_rn / __fmaf_rn would, and is never
// contracted.  Halves the issue slots of the double-float dot products.
__device__ __forceinline__ float2 sub2_rn(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// Double-float sums of two rows at once (the hi and lo parts packed as pairs).
__device__ __forceinline__ void df_add2(float2 &ah, float2 &al, float2 bh, float2 bl) {
  const float2 s = __fadd2_rn(ah, bh);
  const float2 bb = sub2_rn(s, ah);
  const float2 err = __fadd2_rn(sub2_rn(ah, sub2_rn(s, bb)), sub2_rn(bh, bb));
  ah = s;
  al = __fadd2_rn(__fadd2_rn(al, bl), err);
}

// Products of one staged row with v, two adjacent elements per instruction:
// the double-float partial of q_i . v (TwoProd by FMA with the cross terms
// q_hi v_lo and q_lo v_hi, TwoSum into a running pair per lane; the even and
// odd lanes are returned unjoined) and, with CORR, the delayed corrections
// corr += c_i q_i and cv += g_i q_i.  vn = -vh, so -q v_hi needs no negation.
template <bool LO, bool CORR>
__device__ __forceinline__ void row_products(const float4 *slot, float2 cg,
                                             const float2 (&vh)[4], const float2 (&vn)[4],
                                             const float2 (&vl)[4], float2 (&corr)[4],
                                             float2 (&cv)[4], float2 &sh_out, float2 &sl_out) {
  float2 sh = make_float2(0.f, 0.f), sl = make_float2(0.f, 0.f);
  const float2 cf = make_float2(cg.x, cg.x), gf = make_float2(cg.y, cg.y);
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const float4 h4 = slot[u * VEC_THREADS];
    const float4 l4 = LO ? slot[(2 + u) * VEC_THREADS] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int m = 2 * u + p;
      const float2 xa = p ? make_float2(h4.z, h4.w) : make_float2(h4.x, h4.y);
      const float2 xb = p ? make_float2(l4.z, l4.w) : make_float2(l4.x, l4.y);
      if (CORR) {
        corr[m] = __ffma2_rn(cf, xa, corr[m]);
        cv[m] = __ffma2_rn(gf, xa, cv[m]);
      }
      const float2 pn = __fmul2_rn(xa, vn[m]);        // -fl(q_hi v_hi)
      float2 err = __ffma2_rn(xa, vh[m], pn);         // q_hi v_hi - fl(q_hi v_hi), exact
      err = __ffma2_rn(xa, vl[m], err);
      if (LO) err = __ffma2_rn(xb, vh[m], err);
      // TwoSum: sh + fl(q_hi v_hi) = s + e exactly
      const float2 s = sub2_rn(sh, pn);
      const float2 bb = sub2_rn(s, sh);
      const float2 e = sub2_rn(sub2_rn(sh, sub2_rn(s, bb)), __fadd2_rn(pn, bb));
      sh = s;
      sl = __fadd2_rn(__fadd2_rn(sl, e), err);
    }
  }
  sh_out = sh;   // even and odd elements: joined by the caller, two rows at a time
  sl_out = sl;
}

// All rows i = nrows - 1 down to 0 (the newest row first), two per trip.
// Row partials of the block go to dp[i] (one double per row), through a
// transposed butterfly over the warp every two trips (12 shuffles for four
// rows) and a fixed-order sum over the eight warps in shared memory, 32 rows
// at a time.
// cg[i] = (c_i, g_i), read only with CORR.
template <bool LO, bool CORR>
__device__ __forceinline__ void sweep_all_rows(const VecCtx &c, int b, int nrows, int ebase,
                                               const float2 *cg, const float2 (&vh)[4],
                                               const float2 (&vl)[4], float2 (&corr)[4],
                                               float2 (&cv)[4],
                                               float2 (*part)[32][VEC_THREADS / 32],
                                               double *dp, float4 *stg) {
  constexpr int NV = LO ? 4 : 2;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float2 vn[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) vn[m] = make_float2(-vh[m].x, -vh[m].y);
  // N is a multiple of 128, so each 4-element piece of the thread lies wholly
  // inside a row or wholly past its end; pieces past the end read zeros,
  // filled into their slots once
  const bool ok0 = ebase < c.N, ok1 = ebase + 128 < c.N;
  float4 *mine = stg + threadIdx.x;
  if (!ok1) {
    for (int s = 0; s < SW_SLOTS; ++s) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (u == 0 && ok0) continue;
        mine[(s * NV + u) * VEC_THREADS] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (LO) mine[(s * NV + 2 + u) * VEC_THREADS] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
  const size_t rstride = (size_t)c.Bs * c.N;
  const float *hb = c.bhi + (size_t)b * c.N + ebase;
  const float *lb = LO ? c.blo + (size_t)b * c.N + ebase : nullptr;
  // sequence index r (row nrows - 1 - r) into slot s; one commit group per
  // index, empty past the last row
  // shared addresses as 32-bit offsets and the four pieces of a row at
  // immediate offsets from one global and one shared address
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(mine);
  // the lo row sits at a fixed distance from the hi row (flat addresses)
  const uintptr_t dlo = LO ? (uintptr_t)lb - (uintptr_t)hb : 0;
  constexpr int PB = VEC_THREADS * 16;   // bytes between a thread's pieces
  auto stage = [&](int r, int s) {
    if (r < nrows) {
      const float *g = hb + (size_t)(nrows - 1 - r) * rstride;
      const uint32_t sa = sbase + (uint32_t)(s * NV * PB);
      if (ok0) {
        cp_async16_at<0, 0>(sa, g);
        if (LO) cp_async16_at<2 * PB, 0>(sa, reinterpret_cast<const void *>((uintptr_t)g + dlo));
      }
      if (ok1) {
        cp_async16_at<PB, 512>(sa, g);
        if (LO) cp_async16_at<3 * PB, 512>(sa, reinterpret_cast<const void *>((uintptr_t)g + dlo));
      }
    }
    cp_async_commit();
  };
  for (int r = 0; r < SW_SLOTS; ++r) stage(r, r);
  int sc = 0;   // slot of sequence index rs: rs % SW_SLOTS
  for (int t0 = 0; t0 < nrows; t0 += 32) {
    const int nt = min(32, nrows - t0);
    float2 (*pp)[VEC_THREADS / 32] = part[(t0 >> 5) & 1];
    for (int r = 0; r < nt; r += 4) {
      // two trips of two rows each, then one butterfly for the four
      float sh[4], sl[4];
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        const int rs = t0 + r + 2 * hf;   // sequence indices rs, rs + 1
        if (r + 2 * hf >= nt) {         // past the last row (uniform)
          sh[2 * hf] = sl[2 * hf] = sh[2 * hf + 1] = sl[2 * hf + 1] = 0.f;
          continue;
        }
        cp_async_wait<SW_SLOTS - 2>();
        float2 ph[2], pl[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int rq = rs + q;
          if (rq < nrows) {
            const float2 g = CORR ? cg[nrows - 1 - rq] : make_float2(0.f, 0.f);
            row_products<LO, CORR>(mine + (sc + q) * NV * VEC_THREADS, g, vh, vn, vl, corr, cv,
                                   ph[q], pl[q]);
          } else {
            ph[q] = pl[q] = make_float2(0.f, 0.f);
          }
        }
        {
          // join even and odd elements of both rows in one packed sum
          float2 jh = make_float2(ph[0].x, ph[1].x), jl = make_float2(pl[0].x, pl[1].x);
          df_add2(jh, jl, make_float2(ph[0].y, ph[1].y), make_float2(pl[0].y, pl[1].y));
          sh[2 * hf] = jh.x;
          sh[2 * hf + 1] = jh.y;
          sl[2 * hf] = jl.x;
          sl[2 * hf + 1] = jl.y;
        }
        stage(rs + SW_SLOTS, sc);
        stage(rs + SW_SLOTS + 1, sc + 1);
        sc = sc == SW_SLOTS - 2 ? 0 : sc + 2;
      }
      // transposed butterfly over the four rows: across 16 lanes each half
      // keeps two rows (packed), across 8 lanes one; row q ends in lane 8q
      const bool b16 = (lane & 16) != 0, b8 = (lane & 8) != 0;
      float2 kh = b16 ? make_float2(sh[2], sh[3]) : make_float2(sh[0], sh[1]);
      float2 kl = b16 ? make_float2(sl[2], sl[3]) : make_float2(sl[0], sl[1]);
      {
        const float2 oh = b16 ? make_float2(sh[0], sh[1]) : make_float2(sh[2], sh[3]);
        const float2 ol = b16 ? make_float2(sl[0], sl[1]) : make_float2(sl[2], sl[3]);
        const float2 rh = make_float2(__shfl_xor_sync(0xffffffffu, oh.x, 16),
                                      __shfl_xor_sync(0xffffffffu, oh.y, 16));
        const float2 rl = make_float2(__shfl_xor_sync(0xffffffffu, ol.x, 16),
                                      __shfl_xor_sync(0xffffffffu, ol.y, 16));
        df_add2(kh, kl, rh, rl);
      }
      float th = b8 ? kh.y : kh.x, tl = b8 ? kl.y : kl.x;
      {
        const float rh = __shfl_xor_sync(0xffffffffu, b8 ? kh.x : kh.y, 8);
        const float rl = __shfl_xor_sync(0xffffffffu, b8 ? kl.x : kl.y, 8);
        df_add(th, tl, rh, rl);
      }
#pragma unroll
      for (int o = 4; o >= 1; o >>= 1) {
        const float rh = __shfl_xor_sync(0xffffffffu, th, o);
        const float rl = __shfl_xor_sync(0xffffffffu, tl, o);
        df_add(th, tl, rh, rl);
      }
      if ((lane & 7) == 0 && r + (lane >> 3) < nt) pp[r + (lane >> 3)][wid] = make_float2(th, tl);
    }
    // the two tile buffers alternate, so one barrier per tile suffices: tile
    // t + 2 reuses this buffer only after warp 0 passed tile t + 1's barrier
    __syncthreads();
    if (wid == 0 && lane < nt) {
      float hs = 0.f, ls = 0.f;
#pragma unroll
      for (int w = 0; w < VEC_THREADS / 32; ++w) df_add(hs, ls, pp[lane][w].x, pp[lane][w].y);
      dp[nrows - 1 - t0 - lane] = (double)hs + (double)ls;
    }
  }
  cp_async_wait<0>();
}

// Block-wide sum of a float through the double block_sum.
__device__ __forceinline__ float block_sum_f(float v, double *red) {
  return (float)block_sum((double)v, red);
}

template <bool LO, bool F64U>
__global__ void __launch_bounds__(VEC_THREADS, 2) k_sweep_dcgs(VecCtx c, int j) {
  extern __shared__ float4 dyn[];   // row staging ring, then [j] pairs (c_i, g_i)
  float2 *cg = reinterpret_cast<float2 *>(reinterpret_cast<char *>(dyn) + sweep_stage_bytes<LO>());
  __shared__ float2 part[2][32][VEC_THREADS / 32];
  __shared__ double red[VEC_THREADS / 32];
  const int chunk = blockIdx.x, b = blockIdx.y;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int ebase = chunk * VEC_CHUNK + wid * 256 + 4 * lane;
  if (!live_s(c, b, j)) {
    // stopped or padding vector: the contractions see zeros
    if (c.xh != nullptr) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = ebase + 128 * u;
        if (e < c.N) *reinterpret_cast<uint2 *>(c.xh + kblk_bf16(b, e, c.Bs)) = make_uint2(0u, 0u);
      }
    }
    return;
  }
  const double sinv = c.sinv[b], bj = c.betaj[b];
  // alpha~_j = q~_j . C q~_j: from the FP64 contraction's partials, or
  // sum Delta^2 q~^2 + c_K y . bf16(y) on the tensor-core path
  double s = 0.0;
  if (F64U) {
    for (int t = threadIdx.x; t < c.n_mt; t += VEC_THREADS) s += c.alpha_part[(size_t)t * c.Bs + b];
    s *= sinv * sinv;
  } else {
    // the partials of step j (parity j & 1): this kernel writes those of
    // step j + 1 into the other half, so no block can read a sibling's
    // new value
    const float *dq2 = c.dq2_part + (size_t)(j & 1) * c.Bs * c.nchunks;
    double sq = 0.0, sy = 0.0;
    for (int t = threadIdx.x; t < c.nchunks; t += VEC_THREADS)
      sq += (double)dq2[(size_t)b * c.nchunks + t];
    for (int t = threadIdx.x; t < c.n_yb; t += VEC_THREADS)
      sy += (double)c.yy_part[(size_t)b * c.n_yb + t];
    s = sq * sinv * sinv + c.kf * sy;
  }
  const double alpha = block_sum(s, red);
  if (chunk == 0 && threadIdx.x == 0) c.alpha[(size_t)(c.vec0 + b) * c.k + j] = alpha;
  // c_i = h_i / beta_j and g = (T_{j-1} - alpha~) c; the chunk-0 block keeps
  // g in FP64 for the reduction
  {
    const size_t v = (size_t)(c.vec0 + b);
    const double *hb = c.h + (size_t)b * c.kmax1;
    for (int i = threadIdx.x; i < j; i += VEC_THREADS) {
      const double ci = hb[i] * sinv;
      double g = (c.alpha[v * c.k + i] - alpha) * ci;
      if (i >= 1) g = fma(c.beta[v * c.k + i - 1], hb[i - 1] * sinv, g);
      if (i + 1 < j) g = fma(c.beta[v * c.k + i], hb[i + 1] * sinv, g);
      cg[i] = make_float2((float)ci, (float)g);
      if (chunk == 0) c.gq[(size_t)b * c.kmax1 + i] = g;
    }
  }
  __syncthreads();

  const size_t voff = (size_t)b * c.N;
  // v is kept as the float pair (vh, vl), 48 bits: the projections are
  // computed for exactly that vector, and it is what the next step carries.
  // q~_j = w_{j-1} / beta_j is read again after the row loop rather than
  // held in registers through it.
  float vh[8], vl[8], corr[8], cv[8];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int e = ebase + 128 * u;
    double qt[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      vh[4 * u + t] = 0.0f;
      vl[4 * u + t] = 0.0f;
      corr[4 * u + t] = 0.0f;
      cv[4 * u + t] = 0.0f;
    }
    if (e >= c.N) continue;
    const double2 w0 = *reinterpret_cast<const double2 *>(c.wv + voff + e);
    const double2 w1 = *reinterpret_cast<const double2 *>(c.wv + voff + e + 2);
    const double wq[4] = {w0.x, w0.y, w1.x, w1.y};
    double uu[4];
    if (F64U) {
      const double2 a0 = *reinterpret_cast<const double2 *>(c.uC + voff + e);
      const double2 a1 = *reinterpret_cast<const double2 *>(c.uC + voff + e + 2);
      const double av[4] = {a0.x, a0.y, a1.x, a1.y};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        qt[t] = wq[t] * sinv;
        uu[t] = av[t] * sinv;
      }
    } else {
      const float4 uk = *reinterpret_cast<const float4 *>(c.ucd + kblk_f32(b, e, c.Bs));
      const double2 d0 = *reinterpret_cast<const double2 *>(c.Delta2 + e);
      const double2 d1 = *reinterpret_cast<const double2 *>(c.Delta2 + e + 2);
      const double dd[4] = {d0.x, d0.y, d1.x, d1.y};
      const float ku[4] = {uk.x, uk.y, uk.z, uk.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        qt[t] = wq[t] * sinv;
        // C q~ = Delta^2 q~ + c_K Delta^1/2 L L^T Delta^1/2 q~   (Eq. 4)
        uu[t] = fma(dd[t], qt[t], (double)ku[t]);
      }
    }
    double qp[4] = {0.0, 0.0, 0.0, 0.0};
    if (j >= 1) {
      const float4 ph = *reinterpret_cast<const float4 *>(bhi_row(c, j - 1, b) + e);
      const float4 pl = LO ? *reinterpret_cast<const float4 *>(blo_row(c, j - 1, b) + e)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
      qp[0] = (double)ph.x + (double)pl.x;
      qp[1] = (double)ph.y + (double)pl.y;
      qp[2] = (double)ph.z + (double)pl.z;
      qp[3] = (double)ph.w + (double)pl.w;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int m = 4 * u + t;
      const double vd = fma(-bj, qp[t], fma(-alpha, qt[t], uu[t]));
      vh[m] = __double2float_rn(vd);
      vl[m] = __double2float_rn(vd - (double)vh[m]);
    }
  }

  double *dp = c.dot_part + ((size_t)b * c.nchunks + chunk) * c.kmax1;
  {
    float2 vh2[4], vl2[4], corr2[4], cv2[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      vh2[m] = make_float2(vh[2 * m], vh[2 * m + 1]);
      vl2[m] = make_float2(vl[2 * m], vl[2 * m + 1]);
      corr2[m] = make_float2(0.f, 0.f);
      cv2[m] = make_float2(0.f, 0.f);
    }
    sweep_all_rows<LO, true>(c, b, j, ebase, cg, vh2, vl2, corr2, cv2, part, dp, dyn);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      corr[2 * m] = corr2[m].x;
      corr[2 * m + 1] = corr2[m].y;
      cv[2 * m] = cv2[m].x;
      cv[2 * m + 1] = cv2[m].y;
    }
  }

  // q_j into row j of the basis; carried vector, operand and partials
  float *hn = c.bhi + ((size_t)j * c.Bs + b) * c.N;
  float *ln = LO ? c.blo + ((size_t)j * c.Bs + b) * c.N : nullptr;
  double hj = 0.0, nrm = 0.0;
  float dq = 0.0f;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int e = ebase + 128 * u;
    if (e >= c.N) continue;
    float qh4[4], ql4[4];
    double vd[4];
    const double2 w0 = *reinterpret_cast<const double2 *>(c.wv + voff + e);
    const double2 w1 = *reinterpret_cast<const double2 *>(c.wv + voff + e + 2);
    const double wq[4] = {w0.x, w0.y, w1.x, w1.y};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int m = 4 * u + t;
      vd[t] = ((double)vh[m] + (double)vl[m]) - (double)cv[m];   // w_j = v - Q_{j-1} g
      vh[m] = __double2float_rn(vd[t]);
      const double qj = wq[t] * sinv - (double)corr[m];
      qh4[t] = __double2float_rn(qj);
      ql4[t] = __double2float_rn(qj - (double)qh4[t]);
      hj = fma(qj, vd[t], hj);
      nrm = fma(vd[t], vd[t], nrm);
    }
    *reinterpret_cast<float4 *>(hn + e) = make_float4(qh4[0], qh4[1], qh4[2], qh4[3]);
    if (LO) *reinterpret_cast<float4 *>(ln + e) = make_float4(ql4[0], ql4[1], ql4[2], ql4[3]);
    *reinterpret_cast<double2 *>(c.wv + voff + e) = make_double2(vd[0], vd[1]);
    *reinterpret_cast<double2 *>(c.wv + voff + e + 2) = make_double2(vd[2], vd[3]);
    if (c.xh != nullptr) {
      __nv_bfloat162 x01, x23;
      x01.x = __float2bfloat16_rn(c.dsqf[e] * vh[4 * u]);
      x01.y = __float2bfloat16_rn(c.dsqf[e + 1] * vh[4 * u + 1]);
      x23.x = __float2bfloat16_rn(c.dsqf[e + 2] * vh[4 * u + 2]);
      x23.y = __float2bfloat16_rn(c.dsqf[e + 3] * vh[4 * u + 3]);
      uint2 pk;
      pk.x = *reinterpret_cast<uint32_t *>(&x01);
      pk.y = *reinterpret_cast<uint32_t *>(&x23);
      *reinterpret_cast<uint2 *>(c.xh + kblk_bf16(b, e, c.Bs)) = pk;
    }
    if (c.dq2_part != nullptr) {
#pragma unroll
      for (int t = 0; t < 4; ++t) dq = fmaf(c.d2f[e + t] * vh[4 * u + t], vh[4 * u + t], dq);
    }
  }
  hj = block_sum(hj, red);
  nrm = block_sum(nrm, red);
  if (c.dq2_part != nullptr) dq = block_sum_f(dq, red);
  if (threadIdx.x == 0) {
    const size_t pi = (size_t)b * c.nchunks + chunk;
    c.hj_part[pi] = hj;
    c.norm_a[pi] = nrm;
    if (c.dq2_part != nullptr) c.dq2_part[(size_t)((j + 1) & 1) * c.Bs * c.nchunks + pi] = dq;
  }
}

// Per vector: h' = Q_j^T v (fixed-order sums over chunks), the recorded
// alpha_j = alpha~_j + h'_j - h_{j-1}, and beta_{j+1}^2 = ||v||^2 - ||h'||^2.
// Where the projection removes more than half of ||v||^2 the vector is
// flagged for a second pass (the CGS1K criterion) and beta waits for it.
__global__ void __launch_bounds__(256) k_reduce_dcgs(VecCtx c, int j) {
  __shared__ double red[256 / 32];
  __shared__ double hprev;
  const int b = blockIdx.x;
  const int v = c.vec0 + b;
  if (!live_s(c, b, j)) {
    if (threadIdx.x == 0) {
      c.flag2[b] = 0;
      c.sinv[b] = 0.0;
      c.betaj[b] = 0.0;
    }
    return;
  }
  if (threadIdx.x == 0) hprev = j >= 1 ? c.h[(size_t)b * c.kmax1 + j - 1] : 0.0;
  __syncthreads();
  double hh = 0.0;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    double s = 0.0;
    if (i < j) {
      const double *p = c.dot_part + (size_t)b * c.nchunks * c.kmax1 + i;
      for (int ch = 0; ch < c.nchunks; ++ch) s += p[(size_t)ch * c.kmax1];
      s -= c.gq[(size_t)b * c.kmax1 + i];   // the sweep removed Q_{j-1} g
    } else {
      for (int ch = 0; ch < c.nchunks; ++ch) s += c.hj_part[(size_t)b * c.nchunks + ch];
      const size_t ai = (size_t)v * c.k + j;
      const double a = c.alpha[ai] + s - hprev;
      c.alpha[ai] = a;
      c.amax[b] = fmax(c.amax[b], fabs(a));
    }
    c.h[(size_t)b * c.kmax1 + i] = s;
    hh = fma(s, s, hh);
  }
  double nw = 0.0;
  for (int ch = threadIdx.x; ch < c.nchunks; ch += blockDim.x)
    nw += c.norm_a[(size_t)b * c.nchunks + ch];
  hh = block_sum(hh, red);   // the barriers also publish amax[b]
  nw = block_sum(nw, red);
  if (threadIdx.x != 0) return;
  const double rest = nw - hh;
  const int f = rest < 0.5 * nw;
  c.flag2[b] = f;
  if (f) {
    atomicAdd(c.n_second, 1);
    return;
  }
  const double beta = sqrt(fmax(rest, 0.0));
  const bool stop = !(beta > c.tol * c.amax[b]);
  c.beta[(size_t)v * c.k + j] = beta;
  c.betaj[b] = beta;
  if (stop) c.k_eff[v] = j + 1;
  c.sinv[b] = (stop || !(beta > 0.0)) ? 0.0 : 1.0 / beta;
}

// Second pass of the flagged vectors (rare: a large part of v lay in
// span(Q_j)).  Blocks loop over the sub-batch and skip unflagged vectors.
//  update: w' = v - Q_j h' in FP64 from the full float pair (h' need not be
//          small here), with ||w'||^2 partials and the operand written anew;
//  dots:   h'' = Q_j^T w' (double-float);
//  reduce: beta_{j+1}^2 = ||w'||^2 - ||h''||^2, and h'' becomes the delayed
//          update that the next sweep applies.
template <bool LO>
__global__ void __launch_bounds__(VEC_THREADS) k_p2_update_dcgs(VecCtx c, int j) {
  extern __shared__ double hs[];   // [j + 1]
  __shared__ double red[VEC_THREADS / 32];
  const int chunk = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int ebase = chunk * VEC_CHUNK + wid * 256 + 4 * lane;
  for (int b = blockIdx.y; b < c.Bs; b += gridDim.y) {
    if (!c.flag2[b]) continue;   // uniform over the block
    __syncthreads();             // hs of the previous vector is no longer read
    for (int i = threadIdx.x; i <= j; i += VEC_THREADS) hs[i] = c.h[(size_t)b * c.kmax1 + i];
    __syncthreads();
    double r[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) r[m] = 0.0;
    for (int i = 0; i <= j; ++i) {
      const double hc = hs[i];
      const float *qh = bhi_row(c, i, b);
      const float *ql = LO ? blo_row(c, i, b) : nullptr;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = ebase + 128 * u;
        if (e >= c.N) continue;
        const float4 a = *reinterpret_cast<const float4 *>(qh + e);
        const float4 al = LO ? *reinterpret_cast<const float4 *>(ql + e)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
        r[4 * u] = fma(hc, (double)a.x + (double)al.x, r[4 * u]);
        r[4 * u + 1] = fma(hc, (double)a.y + (double)al.y, r[4 * u + 1]);
        r[4 * u + 2] = fma(hc, (double)a.z + (double)al.z, r[4 * u + 2]);
        r[4 * u + 3] = fma(hc, (double)a.w + (double)al.w, r[4 * u + 3]);
      }
    }
    const size_t voff = (size_t)b * c.N;
    double nrm = 0.0;
    float dq = 0.0f;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = ebase + 128 * u;
      if (e >= c.N) continue;
      double w4[4];
      const double2 w0 = *reinterpret_cast<const double2 *>(c.wv + voff + e);
      const double2 w1 = *reinterpret_cast<const double2 *>(c.wv + voff + e + 2);
      w4[0] = w0.x - r[4 * u];
      w4[1] = w0.y - r[4 * u + 1];
      w4[2] = w1.x - r[4 * u + 2];
      w4[3] = w1.y - r[4 * u + 3];
      *reinterpret_cast<double2 *>(c.wv + voff + e) = make_double2(w4[0], w4[1]);
      *reinterpret_cast<double2 *>(c.wv + voff + e + 2) = make_double2(w4[2], w4[3]);
      float f4[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        nrm = fma(w4[t], w4[t], nrm);
        f4[t] = __double2float_rn(w4[t]);
        if (c.dq2_part != nullptr) dq = fmaf(c.d2f[e + t] * f4[t], f4[t], dq);
      }
      if (c.xh != nullptr) {
        __nv_bfloat162 x01, x23;
        x01.x = __float2bfloat16_rn(c.dsqf[e] * f4[0]);
        x01.y = __float2bfloat16_rn(c.dsqf[e + 1] * f4[1]);
        x23.x = __float2bfloat16_rn(c.dsqf[e + 2] * f4[2]);
        x23.y = __float2bfloat16_rn(c.dsqf[e + 3] * f4[3]);
        uint2 pk;
        pk.x = *reinterpret_cast<uint32_t *>(&x01);
        pk.y = *reinterpret_cast<uint32_t *>(&x23);
        *reinterpret_cast<uint2 *>(c.xh + kblk_bf16(b, e, c.Bs)) = pk;
      }
    }
    nrm = block_sum(nrm, red);
    if (c.dq2_part != nullptr) dq = block_sum_f(dq, red);
    if (threadIdx.x == 0) {
      c.norm_b[(size_t)b * c.nchunks + chunk] = nrm;
      if (c.dq2_part != nullptr)
        c.dq2_part[(size_t)((j + 1) & 1) * c.Bs * c.nchunks + (size_t)b * c.nchunks + chunk] = dq;
    }
  }
}

template <bool LO>
__global__ void __launch_bounds__(VEC_THREADS) k_p2_dots_dcgs(VecCtx c, int j) {
  extern __shared__ float4 stg[];   // row staging ring
  __shared__ float2 part[2][32][VEC_THREADS / 32];
  const int chunk = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int ebase = chunk * VEC_CHUNK + wid * 256 + 4 * lane;
  for (int b = blockIdx.y; b < c.Bs; b += gridDim.y) {
    if (!c.flag2[b]) continue;   // uniform over the block
    const size_t voff = (size_t)b * c.N;
    float vh[8], vl[8];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = ebase + 128 * u;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        vh[4 * u + t] = vl[4 * u + t] = 0.0f;
        if (e < c.N) {
          const double x = c.wv[voff + e + t];
          vh[4 * u + t] = __double2float_rn(x);
          vl[4 * u + t] = __double2float_rn(x - (double)vh[4 * u + t]);
        }
      }
    }
    float2 vh2[4], vl2[4], unused[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      vh2[m] = make_float2(vh[2 * m], vh[2 * m + 1]);
      vl2[m] = make_float2(vl[2 * m], vl[2 * m + 1]);
      unused[m] = make_float2(0.f, 0.f);
    }
    double *dp = c.dot_part + ((size_t)b * c.nchunks + chunk) * c.kmax1;
    __syncthreads();   // the tile buffers of the previous vector are free
    sweep_all_rows<LO, false>(c, b, j + 1, ebase, nullptr, vh2, vl2, unused, unused, part, dp,
                              stg);
  }
}

__global__ void __launch_bounds__(256) k_p2_reduce_dcgs(VecCtx c, int j) {
  __shared__ double red[256 / 32];
  const int b = blockIdx.x;
  const int v = c.vec0 + b;
  if (!c.flag2[b]) return;
  double hh = 0.0;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const double *p = c.dot_part + (size_t)b * c.nchunks * c.kmax1 + i;
    double s = 0.0;
    for (int ch = 0; ch < c.nchunks; ++ch) s += p[(size_t)ch * c.kmax1];
    c.h[(size_t)b * c.kmax1 + i] = s;
    hh = fma(s, s, hh);
  }
  double nw = 0.0;
  for (int ch = threadIdx.x; ch < c.nchunks; ch += blockDim.x)
    nw += c.norm_b[(size_t)b * c.nchunks + ch];
  hh = block_sum(hh, red);
  nw = block_sum(nw, red);
  if (threadIdx.x != 0) return;
  const double beta = sqrt(fmax(nw - hh, 0.0));
  const bool stop = !(beta > c.tol * c.amax[b]);
  c.beta[(size_t)v * c.k + j] = beta;
  c.betaj[b] = beta;
  if (stop) c.k_eff[v] = j + 1;
  c.sinv[b] = (stop || !(beta > 0.0)) ? 0.0 : 1.0 / beta;
}

// Dynamic shared memory above 48 KB needs the attribute, set once per kernel.
template <class K>
static void allow_smem(K kern, size_t bytes) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <bool LO, bool F64U>
static void sweep_one(const VecCtx &c, int j, cudaStream_t st) {
  static bool attr = false;
  constexpr size_t max_sh = sweep_stage_bytes<LO>() + (size_t)4096 * sizeof(float2);
  if (!attr) {
    allow_smem(k_sweep_dcgs<LO, F64U>, max_sh);
    attr = true;
  }
  const size_t sh = sweep_stage_bytes<LO>() + (size_t)(j > 0 ? j : 1) * sizeof(float2);
  k_sweep_dcgs<LO, F64U><<<dim3(c.nchunks, c.Bs), VEC_THREADS, sh, st>>>(c, j);
}

void launch_sweep_dcgs(const VecCtx &c, int j, cudaStream_t st) {
  const bool lo = c.blo != nullptr, f64u = c.uC != nullptr;
  if (lo && f64u)
    sweep_one<true, true>(c, j, st);
  else if (lo)
    sweep_one<true, false>(c, j, st);
  else if (f64u)
    sweep_one<false, true>(c, j, st);
  else
    sweep_one<false, false>(c, j, st);
}
void launch_reduce_dcgs(const VecCtx &c, int j, cudaStream_t st) {
  k_reduce_dcgs<<<c.Bs, 256, 0, st>>>(c, j);
}
void launch_pass2_dcgs(const VecCtx &c, int j, cudaStream_t st) {
  const dim3 grid(c.nchunks, c.Bs < 16 ? c.Bs : 16);
  const size_t sh = (size_t)(j + 1) * sizeof(double);
  static bool attr = false;
  if (!attr) {
    allow_smem(k_p2_dots_dcgs<true>, sweep_stage_bytes<true>());
    allow_smem(k_p2_dots_dcgs<false>, sweep_stage_bytes<false>());
    attr = true;
  }
  if (c.blo != nullptr) {
    k_p2_update_dcgs<true><<<grid, VEC_THREADS, sh, st>>>(c, j);
    k_p2_dots_dcgs<true><<<grid, VEC_THREADS, sweep_stage_bytes<true>(), st>>>(c, j);
  } else {
    k_p2_update_dcgs<false><<<grid, VEC_THREADS, sh, st>>>(c, j);
    k_p2_dots_dcgs<false><<<grid, VEC_THREADS, sweep_stage_bytes<false>(), st>>>(c, j);
  }
  k_p2_reduce_dcgs<<<c.Bs, 256, 0, st>>>(c, j);
}

static dim3 grid_s(const VecCtx &c) { return dim3(c.nchunks, c.Bs); }

void launch_dots_split(const VecCtx &c, int j, int pass, cudaStream_t st) {
  if (pass == 1)
    k_dots_split<1><<<grid_s(c), VEC_THREADS, 0, st>>>(c, j);
  else
    k_dots_split<2><<<grid_s(c), VEC_THREADS, 0, st>>>(c, j);
}
void launch_reduce_dots_split(const VecCtx &c, int j, int pass, cudaStream_t st) {
  k_reduce_dots_split<<<c.Bs, 256, 0, st>>>(c, j, pass);
}
void launch_update_split(const VecCtx &c, int j, int pass, cudaStream_t st) {
  const size_t sh = (size_t)c.kmax1 * sizeof(float);
  if (pass == 1)
    k_update_split<1><<<grid_s(c), VEC_THREADS, sh, st>>>(c, j);
  else
    k_update_split<2><<<grid_s(c), VEC_THREADS, sh, st>>>(c, j);
}
void launch_start_split(const VecCtx &c, cudaStream_t st) {
  k_start_split<<<grid_s(c), VEC_THREADS, 0, st>>>(c);
}

}  // namespace lgw
