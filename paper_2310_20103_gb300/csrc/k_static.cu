// The static part of the self-energy and the density-fitting front end.
//
// Exchange (text after Eq. 5): Sigma^ex_t = -sum_v (vt|vt).  The pair factors
// share L's metric-folded form, (pq|rs) = sum_mu B_pq,mu B_rs,mu, so with the
// factors M[t][m][:] of the request (vt|vt) = sum_mu M[t][v][mu]^2 for the
// occupied orbitals v of the summed set.
//
// Density fitting: with fitting coefficients C_ab,mu and the Coulomb metric
// V_mu,nu = (mu|nu), (ab|cd) = sum C_ab,mu V_mu,nu C_cd,nu; V = R R^T
// (Cholesky, R lower) gives the factors B = C R.  FP64 throughout.
#include <algorithm>

#include "lgw_internal.cuh"

namespace lgw {

__global__ void k_sigma_x(const double *__restrict__ M, int n_m, int n_aux,
                          const int *__restrict__ m_idx, int n_v, double *__restrict__ out) {
  __shared__ double red[8];
  const int t = blockIdx.x;
  double s = 0.0;
  for (int mi = 0; mi < n_m; ++mi) {
    if (m_idx[mi] >= n_v) continue;
    const double *row = M + ((size_t)t * n_m + mi) * n_aux;
    for (int mu = threadIdx.x; mu < n_aux; mu += blockDim.x) s = fma(row[mu], row[mu], s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[t] = -s;
}

// --------------------------------------------------------------------------
// Blocked right-looking Cholesky, NB x NB blocks, in place on the lower
// triangle of a [n][n] row-major matrix.
// --------------------------------------------------------------------------
constexpr int NB = 64;

// factor the diagonal block at (j0, j0); one CTA of NB threads, row i per thread
__global__ void __launch_bounds__(NB) k_potrf_diag(double *A, int n, int j0, unsigned *status) {
  __shared__ double blk[NB][NB + 1];
  const int i = threadIdx.x;
  const int nb = min(NB, n - j0);
  for (int c = 0; c < nb; ++c) blk[i][c] = (i < nb) ? A[(size_t)(j0 + i) * n + j0 + c] : 0.0;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (i == j) {
      double d = blk[j][j];
      for (int p = 0; p < j; ++p) d = fma(-blk[j][p], blk[j][p], d);
      if (!(d > 0.0)) {
        atomicOr(status, ST_NOT_SPD);
        d = 1.0;
      }
      blk[j][j] = sqrt(d);
    }
    __syncthreads();
    if (i > j && i < nb) {
      double x = blk[i][j];
      for (int p = 0; p < j; ++p) x = fma(-blk[i][p], blk[j][p], x);
      blk[i][j] = x / blk[j][j];
    }
    __syncthreads();
  }
  if (i < nb)
    for (int c = 0; c <= i; ++c) A[(size_t)(j0 + i) * n + j0 + c] = blk[i][c];
}

// rows below the diagonal block: L_i = A_i L_jj^{-T} (forward substitution,
// one row per thread)
__global__ void k_trsm_panel(double *A, int n, int j0) {
  __shared__ double Ljj[NB][NB + 1];
  const int nb = min(NB, n - j0);
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    const int r = idx / NB, c = idx % NB;
    Ljj[r][c] = (r < nb && c <= r) ? A[(size_t)(j0 + r) * n + j0 + c] : 0.0;
  }
  __syncthreads();
  const int i = j0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double *row = A + (size_t)i * n + j0;
  for (int c = 0; c < nb; ++c) {
    double v = row[c];
    for (int p = 0; p < c; ++p) v = fma(-row[p], Ljj[c][p], v);
    row[c] = v / Ljj[c][c];
  }
}

// trailing update A[i][j] -= sum_p L[i][j0+p] L[j][j0+p] for i, j >= j0+nb,
// lower triangle (64 x 64 output tiles, 4 x 4 per thread, the panel in
// 16-column slices)
__global__ void __launch_bounds__(256) k_syrk_update(double *A, int n, int j0, int nb) {
  const int t0 = j0 + nb;
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  __shared__ double Xs[16][65];
  __shared__ double Ys[16][65];
  const int i0 = t0 + bi * 64, jj0 = t0 + bj * 64;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  double acc[4][4] = {};
  for (int p0 = 0; p0 < nb; p0 += 16) {
#pragma unroll
    for (int rep = 0; rep < 4; ++rep) {
      const int idx = t + 256 * rep;
      const int p = idx & 15, r = idx >> 4;
      const bool pk = p0 + p < nb;
      Xs[p][r] = (i0 + r < n && pk) ? A[(size_t)(i0 + r) * n + j0 + p0 + p] : 0.0;
      Ys[p][r] = (jj0 + r < n && pk) ? A[(size_t)(jj0 + r) * n + j0 + p0 + p] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < 16; ++p) {
      double xa[4], yb[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) xa[q] = Xs[p][ty + 16 * q];
#pragma unroll
      for (int q = 0; q < 4; ++q) yb[q] = Ys[p][tx + 16 * q];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[q][w] = fma(xa[q], yb[w], acc[q][w]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + ty + 16 * q;
    if (i >= n) continue;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int j = jj0 + tx + 16 * w;
      if (j < n && j <= i) A[(size_t)i * n + j] -= acc[q][w];
    }
  }
}

__global__ void k_zero_upper(double *A, int n) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  if (j > i) A[idx] = 0.0;
}

// Cm[M][N] = Am[M][K] Bm[K][N], row-major, FP64 (64 x 64 tiles)
__global__ void __launch_bounds__(256) k_gemm_nn_f64(const double *__restrict__ Am,
                                                     const double *__restrict__ Bm, int M, int N,
                                                     int K, double *__restrict__ Cm) {
  __shared__ double As[16][65];
  __shared__ double Bs[16][65];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
    for (int rep = 0; rep < 4; ++rep) {
      const int idx = t + 256 * rep;
      const int kk = idx & 15, m = idx >> 4;          // A tile: 64 rows x 16
      As[kk][m] = (m0 + m < M && k0 + kk < K) ? Am[(size_t)(m0 + m) * K + k0 + kk] : 0.0;
      const int nn = idx & 63, k2 = idx >> 6;         // B tile: 16 x 64 cols
      Bs[k2][nn] = (k0 + k2 < K && n0 + nn < N) ? Bm[(size_t)(k0 + k2) * N + n0 + nn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nn = n0 + tx + 16 * j;
      if (nn < N) Cm[(size_t)m * N + nn] = acc[i][j];
    }
  }
}

// ----------------------------------------------------------------------------
void launch_sigma_x(const double *M, int n_t, int n_m, int n_aux, const int *m_idx, int n_v,
                    double *out, cudaStream_t st) {
  if (n_t > 0) k_sigma_x<<<n_t, 256, 0, st>>>(M, n_m, n_aux, m_idx, n_v, out);
}

int launch_cholesky(double *A, int n, unsigned *status, cudaStream_t st) {
  int launches = 0;
  for (int j0 = 0; j0 < n; j0 += NB) {
    const int nb = std::min(NB, n - j0);
    k_potrf_diag<<<1, NB, 0, st>>>(A, n, j0, status);
    ++launches;
    const int rest = n - j0 - nb;
    if (rest > 0) {
      k_trsm_panel<<<(rest + 127) / 128, 128, 0, st>>>(A, n, j0);
      const int tiles = (rest + 63) / 64;
      k_syrk_update<<<dim3(tiles, tiles), 256, 0, st>>>(A, n, j0, nb);
      launches += 2;
    }
  }
  k_zero_upper<<<(unsigned)(((size_t)n * n + 255) / 256), 256, 0, st>>>(A, n);
  return launches + 1;
}

void launch_gemm_nn_f64(const double *A, const double *B, int M, int N, int K, double *C,
                        cudaStream_t st) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  k_gemm_nn_f64<<<grid, 256, 0, st>>>(A, B, M, N, K, C);
}

}  // namespace lgw
