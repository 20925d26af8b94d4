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
    }
    live = beta > 0.0;
    inv = sinv;
  } else if (chunk == 0 && threadIdx.x == 0) {
    c.betaj[b] = 0.0;
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
