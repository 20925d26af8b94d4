// System preparation: pair energies (Eq. 2-4) and the operand copies of L.
#include "lgw_internal.cuh"

namespace lgw {

// Delta_vc = eps_c - eps_v with vc = v * n_c + c (A - B of Eq. 2-3), its
// square root (the factor of |P_tm>, text after Eq. 8) and square (Eq. 4).
// The padding tail [n_vc, N) is zero so padded vectors stay zero.
__global__ void k_pair_energies(const double *__restrict__ eps, int n_v, int n_c, int n_vc, int N,
                                double kf, double *Delta, double *dsq, double *Delta2,
                                double *cd, float *dsqf, float *d2f, float *d2lo, float *cdf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double D = 0.0;
  if (i < n_vc) {
    int v = i / n_c, c = i - v * n_c;
    D = eps[n_v + c] - eps[v];
  }
  double s = D > 0.0 ? sqrt(D) : 0.0;
  Delta[i] = D;
  dsq[i] = s;
  Delta2[i] = D * D;
  cd[i] = kf * s;
  dsqf[i] = (float)s;
  d2f[i] = (float)(D * D);
  d2lo[i] = (float)(D * D - (double)d2f[i]);
  cdf[i] = (float)(kf * s);
}

__global__ void k_check_delta(const double *__restrict__ Delta, int n_vc, unsigned *status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_vc && !(Delta[i] > 0.0)) atomicOr(status, ST_NOT_SPD);
}

// L [n_vc][n_aux] -> L64 [N][A], zero padded.
__global__ void k_pad_L(const double *__restrict__ L, int n_vc, int n_aux, int N, int A,
                        double *__restrict__ L64) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = (int64_t)N * A;
  for (; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(idx / A), c = (int)(idx - (int64_t)r * A);
    L64[idx] = (r < n_vc && c < n_aux) ? L[(int64_t)r * n_aux + c] : 0.0;
  }
}

// BF16 copies from L [nr][nc] (row stride ld), zero padded to [N][A]:
// Lb = bf16(L) [N][A], Ltb = bf16(L)^T [A][N] (K-block-major) and Lb_lo = bf16(L - bf16(L)),
// through a 32x32 shared-memory transpose tile so both writes are coalesced.
__global__ void k_quantize_L(const double *__restrict__ src, int ld, int nr, int nc, int N, int A,
                             __nv_bfloat16 *__restrict__ Lb, __nv_bfloat16 *__restrict__ Ltb,
                             __nv_bfloat16 *__restrict__ Lb_lo) {
  __shared__ __nv_bfloat16 tile[32][33];
  int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  for (int rr = ty; rr < 32; rr += 8) {
    int r = r0 + rr, c = c0 + tx;
    __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
    if (r < N && c < A) {
      const double x = (r < nr && c < nc) ? src[(int64_t)r * ld + c] : 0.0;
      v = __double2bfloat16(x);
      Lb[(int64_t)r * A + c] = v;
      Lb_lo[(int64_t)r * A + c] = __double2bfloat16(x - (double)__bfloat162float(v));
    }
    tile[rr][tx] = v;
  }
  __syncthreads();
  for (int cc = ty; cc < 32; cc += 8) {
    int c = c0 + cc, r = r0 + tx;
    if (r < N && c < A) Ltb[kblk_bf16(c, r, A)] = tile[tx][cc];
  }
}

void launch_pair_energies(const SysDev &s, cudaStream_t st) {
  int th = 256, bl = (s.N + th - 1) / th;
  k_pair_energies<<<bl, th, 0, st>>>(s.eps, s.n_v, s.n_c, s.n_vc, s.N, s.kf, s.Delta, s.dsq,
                                     s.Delta2, s.cd, s.dsqf, s.d2f, s.d2lo, s.cdf);
}

void launch_check_delta(const SysDev &s, unsigned *status, cudaStream_t st) {
  int th = 256, bl = (s.n_vc + th - 1) / th;
  k_check_delta<<<bl, th, 0, st>>>(s.Delta, s.n_vc, status);
}

void launch_pad_L(const double *L, const SysDev &s, cudaStream_t st) {
  int64_t total = (int64_t)s.N * s.A;
  int th = 256;
  int64_t bl = (total + th - 1) / th;
  if (bl > 152 * 64) bl = 152 * 64;
  k_pad_L<<<(int)bl, th, 0, st>>>(L, s.n_vc, s.n_aux, s.N, s.A, s.L64);
}

void launch_quantize_L(const double *src, int ld, int nr, int nc, const SysDev &s,
                       cudaStream_t st) {
  dim3 grid((s.A + 31) / 32, (s.N + 31) / 32);
  k_quantize_L<<<grid, 256, 0, st>>>(src, ld, nr, nc, s.N, s.A, s.Lb, s.Ltb, s.Lb_lo);
}

}  // namespace lgw
