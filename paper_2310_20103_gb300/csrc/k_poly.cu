// Polynomial variant: Lanczos on D = p_g(C) ~ C^1/2 (the paper's form after
// Eq. 12; the fit p_g of sqrt on the spectral interval [lo, hi] of C is the
// Chebyshev interpolant, p_g(x) = sum_k c_k T_k(t), t = (2x - hi - lo)/(hi - lo)).
// One Lanczos step applies D by Clenshaw's recurrence in S = a_s C + b_s I,
// a_s = 2 / (hi - lo), b_s = -(hi + lo) / (hi - lo):
//   b_g = c_g q,   b_k = c_k q + 2 S b_{k+1} - b_{k+2}  (k = g-1 .. 1),
//   D q = c_0 q + S b_1 - b_2,
// so g applications of C (two contractions each) per step.  These kernels
// are the vector passes between the contractions, FP64; the products C b
// arrive either complete in FP64 (T = Delta^2 b + c_K Delta^1/2 L L^T
// Delta^1/2 b) or, from the tensor cores, as ucd = c_K Delta^1/2 (L y) in FP32
// with Delta^2 b added here.  The continued fractions then use D's
// tridiagonal directly (Eq. 14): Sigma_tm = (G(-eta z) - G(0)) / z.
#include "lgw_internal.cuh"

namespace lgw {

__device__ __forceinline__ int poly_elem_base(int chunk) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  return chunk * VEC_CHUNK + wid * 256 + 2 * lane;
}

// C b at element pair e of vector b (FP64 product T [Bs][N], or the FP32
// coupling ucd (kblk_f32 over Bs = gridDim.y vectors) + Delta^2 b)
__device__ __forceinline__ double2 cb_pair(const double *T, const float *ucd, const double *Delta2,
                                           const double2 b1, int b, int e) {
  if (T) return *reinterpret_cast<const double2 *>(T + e);   // T offset to vector b
  const float2 u = *reinterpret_cast<const float2 *>(ucd + kblk_f32(b, e, gridDim.y));
  return make_double2(fma(Delta2[e], b1.x, (double)u.x), fma(Delta2[e + 1], b1.y, (double)u.y));
}

// out = ck q + 2 (a_s C b1 + b_s b1) - b2   (b1, b2 may be NULL: zero);
// xh = bf16(Delta^1/2 out) for the next tensor-core product (or NULL).
__global__ void __launch_bounds__(VEC_THREADS) k_cheb_step(PolyStep p) {
  const int chunk = blockIdx.x, b = blockIdx.y;
  const size_t voff = (size_t)b * p.N;
  const int e0 = poly_elem_base(chunk);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    if (e >= p.N) continue;
    const size_t o = voff + e;
    const double2 q = *reinterpret_cast<const double2 *>(p.q + o);
    double2 r = make_double2(p.ck * q.x, p.ck * q.y);
    if (p.b1) {
      const double2 b1 = *reinterpret_cast<const double2 *>(p.b1 + o);
      const double2 t = cb_pair(p.T ? p.T + voff : nullptr, p.ucd, p.Delta2, b1, b, e);
      r.x = fma(2.0 * p.as, t.x, fma(2.0 * p.bs, b1.x, r.x));
      r.y = fma(2.0 * p.as, t.y, fma(2.0 * p.bs, b1.y, r.y));
    }
    if (p.b2) {
      const double2 b2 = *reinterpret_cast<const double2 *>(p.b2 + o);
      r.x -= b2.x;
      r.y -= b2.y;
    }
    *reinterpret_cast<double2 *>(p.out + o) = r;
    if (p.xh) {
      __nv_bfloat162 x2;
      x2.x = __float2bfloat16_rn(p.dsqf[e] * (float)r.x);
      x2.y = __float2bfloat16_rn(p.dsqf[e + 1] * (float)r.y);
      // K-block-major over the Bs = gridDim.y vectors of the launch
      *reinterpret_cast<__nv_bfloat162 *>(p.xh + kblk_bf16(b, e, gridDim.y)) = x2;
    }
  }
}

// w = c_0 q + a_s C b1 + b_s b1 - b2 - beta_j q_{j-1}, and the per-chunk
// partials of alpha_j = q . w into alpha_part[chunk][b].
__global__ void __launch_bounds__(VEC_THREADS) k_cheb_final(PolyStep p, const double *qprev,
                                                            const double *betaj, double *w,
                                                            double *alpha_part, int Bs) {
  __shared__ double red[VEC_THREADS / 32];
  const int chunk = blockIdx.x, b = blockIdx.y;
  const size_t voff = (size_t)b * p.N;
  const int e0 = poly_elem_base(chunk);
  const double bj = betaj[b];
  double ap = 0.0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + u * 64;
    if (e >= p.N) continue;
    const size_t o = voff + e;
    const double2 q = *reinterpret_cast<const double2 *>(p.q + o);
    const double2 b1 = *reinterpret_cast<const double2 *>(p.b1 + o);
    const double2 t = cb_pair(p.T ? p.T + voff : nullptr, p.ucd, p.Delta2, b1, b, e);
    double2 r;
    r.x = fma(p.as, t.x, fma(p.bs, b1.x, p.ck * q.x));
    r.y = fma(p.as, t.y, fma(p.bs, b1.y, p.ck * q.y));
    if (p.b2) {
      const double2 b2 = *reinterpret_cast<const double2 *>(p.b2 + o);
      r.x -= b2.x;
      r.y -= b2.y;
    }
    if (qprev) {
      const double2 qp = *reinterpret_cast<const double2 *>(qprev + o);
      r.x = fma(-bj, qp.x, r.x);
      r.y = fma(-bj, qp.y, r.y);
    }
    *reinterpret_cast<double2 *>(w + o) = r;
    ap = fma(q.x, r.x, fma(q.y, r.y, ap));
  }
  ap = block_sum(ap, red);
  if (threadIdx.x == 0) alpha_part[(size_t)chunk * Bs + b] = ap;
}

// Haydock coefficients of D's tridiagonal for the continued fractions:
// a = alpha (used in place), b2 = beta^2, w0 = beta0^2, depth k_eff, and
// G(0) = <P|(0 - D_L)^-1|P> (real: D_L is positive definite).
__global__ void k_poly_prep(const double *__restrict__ alpha, const double *__restrict__ beta,
                            const double *__restrict__ beta0, const int *__restrict__ k_eff,
                            int B, int k, JacobiBufs jb, unsigned *status) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= B) return;
  const int n = k_eff[v];
  jb.n[v] = n;
  const double W = beta0[v] * beta0[v];
  jb.w0[v] = W;
  double *b2 = jb.b2 + (size_t)v * k;
  for (int i = 0; i < k; ++i) {
    const double x = (i + 1 < n) ? beta[(size_t)v * k + i] : 0.0;
    b2[i] = x * x;
  }
  if (jb.g0 == nullptr) return;   // Tamm-Dancoff fractions need no G(0)
  if (n <= 0) {
    jb.g0[v] = 0.0;
    return;
  }
  // bottom-up at zeta = 0: t_i = -a_i - b2_i / t_{i+1}, all < 0 for an SPD D_L
  const double *a = alpha + (size_t)v * k;
  double t = -a[n - 1];
  for (int i = n - 2; i >= 0; --i) t = -a[i] - b2[i] / t;
  if (!(t < 0.0)) atomicOr(status, ST_NOT_SPD);
  jb.g0[v] = W / t;
}

void launch_cheb_step(const PolyStep &p, int nchunks, int Bs, cudaStream_t st) {
  k_cheb_step<<<dim3(nchunks, Bs), VEC_THREADS, 0, st>>>(p);
}
void launch_cheb_final(const PolyStep &p, const double *qprev, const double *betaj, double *w,
                       double *alpha_part, int nchunks, int Bs, cudaStream_t st) {
  k_cheb_final<<<dim3(nchunks, Bs), VEC_THREADS, 0, st>>>(p, qprev, betaj, w, alpha_part, Bs);
}
void launch_poly_prep(const double *alpha, const double *beta, const double *beta0,
                      const int *k_eff, int B, int k, JacobiBufs jb, unsigned *status,
                      cudaStream_t st) {
  k_poly_prep<<<(B + 127) / 128, 128, 0, st>>>(alpha, beta, beta0, k_eff, B, k, jb, status);
}

// Tamm-Dancoff view of a system: the Casida arrays of A = Delta + c L L^T
// take the places of those of C (Delta^1/2 -> 1, Delta^2 -> Delta,
// c_K Delta^1/2 -> c), zero in the padding.
__global__ void k_tda_view(const double *__restrict__ Delta, int n_vc, int N, double c,
                           double *ones, double *cd, float *onesf, float *d2f, float *d2lo,
                           float *cdf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const bool real = i < n_vc;
  ones[i] = real ? 1.0 : 0.0;
  cd[i] = real ? c : 0.0;
  onesf[i] = real ? 1.0f : 0.0f;
  d2f[i] = (float)Delta[i];
  d2lo[i] = (float)(Delta[i] - (double)d2f[i]);
  cdf[i] = real ? (float)c : 0.0f;
}

// Sigma_tt' = (Sigma[b_t + b_t'] - Sigma[b_t - b_t']) / 4: virtual requests
// 2i and 2i+1 of pair i carry the rows of t + t' and t - t'.
__global__ void k_pol_rows(const double *__restrict__ src, int n_m, int len,
                           const int *__restrict__ pairs, int n_pairs, double *__restrict__ dst) {
  const size_t row_len = (size_t)n_m * len;
  const size_t n = (size_t)n_pairs * 2 * row_len;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t r = idx / row_len, e = idx % row_len;
    const int i = (int)(r / 2);
    const double a = src[(size_t)pairs[2 * i] * row_len + e];
    const double b = src[(size_t)pairs[2 * i + 1] * row_len + e];
    dst[idx] = (r % 2 == 0) ? a + b : a - b;
  }
}

__global__ void k_pol_combine(const double *__restrict__ sig2, int n_pairs, int n_freq,
                              double *__restrict__ out) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t per = (size_t)n_freq * 2;
  if (idx >= (size_t)n_pairs * per) return;
  const size_t i = idx / per, e = idx % per;
  out[idx] = 0.25 * (sig2[(2 * i) * per + e] - sig2[(2 * i + 1) * per + e]);
}

void launch_tda_view(const double *Delta, int n_vc, int N, double c, double *ones, double *cd,
                     float *onesf, float *d2f, float *d2lo, float *cdf, cudaStream_t st) {
  k_tda_view<<<(N + 255) / 256, 256, 0, st>>>(Delta, n_vc, N, c, ones, cd, onesf, d2f, d2lo,
                                               cdf);
}
void launch_pol_rows(const double *src, int n_m, int len, const int *pairs, int n_pairs,
                     double *dst, cudaStream_t st) {
  const size_t n = (size_t)n_pairs * 2 * n_m * len;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (n) k_pol_rows<<<(unsigned)blocks, 256, 0, st>>>(src, n_m, len, pairs, n_pairs, dst);
}
void launch_pol_combine(const double *sig2, int n_pairs, int n_freq, double *out,
                        cudaStream_t st) {
  const size_t n = (size_t)n_pairs * n_freq * 2;
  if (n) k_pol_combine<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sig2, n_pairs, n_freq, out);
}

}  // namespace lgw
