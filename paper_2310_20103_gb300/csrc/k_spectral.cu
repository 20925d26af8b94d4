// Spectral map of each Lanczos tridiagonal (Eq. 12-14), FP64.
//
// A k-step Lanczos on C from b gives T_k whose Gauss rule (nodes theta_j,
// weights ||b||^2 u_1j^2, u_1j the first components of T_k's eigenvectors)
// reproduces b^T f(C) b for polynomials f of degree < 2k.  Eq. 12 needs
// f(C) = C^-1/2 (z + eta C^1/2)^-1, i.e. the resolvent of D = C^1/2 with the
// weights divided by Omega:  Sigma_tm(omega) = -eta G(-eta z),
//   G(zeta) = sum_j wt_j / (zeta - Omega_j),  Omega_j = sqrt(theta_j),
//   wt_j = ||b||^2 u_1j^2 / Omega_j.
// The continued fraction of Eq. 14 for G needs the Jacobi matrix of this
// discrete measure; it is rebuilt here from (Omega_j, wt_j) by inserting the
// nodes one at a time and chasing the bulge with plane rotations (the
// Rutishauser / Gragg-Harrod reconstruction, O(k^2), orthogonal, stable).
//
// One thread per start vector; the tridiagonal, its first eigenvector row
// and the Jacobi matrix live in per-vector scratch rows of length k.
#include "lgw_internal.cuh"

namespace lgw {

// Plane rotation applied symmetrically to rows/cols (i, i+1) of a symmetric
// tridiagonal with diagonal d and off-diagonal e (e[i] couples i, i+1).
__device__ __forceinline__ void rot_sym(double c, double s, double *d, double *e, int i) {
  const double a = d[i], bb = e[i], cc = d[i + 1];
  const double cs = c * s, c2 = c * c, s2 = s * s;
  d[i] = c2 * a + 2.0 * cs * bb + s2 * cc;
  d[i + 1] = s2 * a - 2.0 * cs * bb + c2 * cc;
  e[i] = cs * (cc - a) + (c2 - s2) * bb;
}

// Givens pair (c, s) with c x + s z = r >= 0, -s x + c z = 0, from one
// reciprocal square root (no FP64 division: GB300 runs FP64 at 1/58 rate).
__device__ __forceinline__ void givens(double x, double z, double &c, double &s, double &r) {
  const double r2 = fma(x, x, z * z);
  if (r2 > 0.0) {
    const double inv = rsqrt(r2);
    c = x * inv;
    s = z * inv;
    r = r2 * inv;
  } else {
    c = 1.0;
    s = 0.0;
    r = 0.0;
  }
}

// Eigenvalues of the symmetric tridiagonal (d[0..n), e[0..n-1)) and the first
// row u of its eigenvector matrix, by implicit symmetric QR steps with the
// Wilkinson shift (Golub & Van Loan, implicit symmetric QR).  On return d
// holds the eigenvalues (unordered) and u the first components.
__device__ bool tridiag_eig_first_row(double *d, double *e, double *u, int n) {
  const double eps = 2.220446049250313e-16;
  for (int i = 0; i < n; ++i) u[i] = (i == 0) ? 1.0 : 0.0;
  if (n > 0) e[n - 1] = 0.0;
  int hi = n - 1;
  int iter = 0;
  const int max_iter = 60 * n + 60;
  while (hi > 0) {
    if (fabs(e[hi - 1]) <= eps * (fabs(d[hi - 1]) + fabs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && fabs(e[lo - 1]) > eps * (fabs(d[lo - 1]) + fabs(d[lo]))) --lo;
    if (lo > 0) e[lo - 1] = 0.0;
    if (++iter > max_iter) return false;
    // Wilkinson shift: eigenvalue of the trailing 2x2 block nearer d[hi]
    const double dl = 0.5 * (d[hi - 1] - d[hi]);
    const double bb = e[hi - 1];
    const double den = dl + copysign(hypot(dl, bb), dl != 0.0 ? dl : 1.0);
    const double mu = d[hi] - bb * bb / den;
    double x = d[lo] - mu, z = e[lo];
    for (int kk = lo; kk < hi; ++kk) {
      double c, s, r;
      givens(x, z, c, s, r);
      if (kk > lo) e[kk - 1] = r;
      rot_sym(c, s, d, e, kk);
      if (kk + 1 < hi) {
        const double bulge = s * e[kk + 1];
        e[kk + 1] *= c;
        x = e[kk];
        z = bulge;
      }
      const double u0 = u[kk], u1 = u[kk + 1];
      u[kk] = c * u0 + s * u1;
      u[kk + 1] = -s * u0 + c * u1;
    }
  }
  return true;
}

// Jacobi matrix (a[0..n), off-diagonal squares b2[0..n-1)) and total weight
// of the discrete measure sum_j wt_j delta(x - x_j), n = number of nodes.
// Node j is added as a new leading row with start-vector weight wt_j; one
// rotation in plane (0,1) folds it into the start vector and the bulge it
// leaves is chased to the bottom.  b holds the off-diagonal (not squared)
// during the build.
__device__ double jacobi_from_nodes(const double *x, const double *wt, int n, double *a, double *b) {
  if (n <= 0) return 0.0;
  a[0] = x[0];
  double W = wt[0];
  int m = 1;
  for (int jn = 1; jn < n; ++jn) {
    for (int i = m; i >= 1; --i) a[i] = a[i - 1];
    for (int i = m - 1; i >= 1; --i) b[i] = b[i - 1];
    a[0] = x[jn];
    b[0] = 0.0;
    const double wj = wt[jn];
    double c = 1.0, s = 0.0;
    if (W + wj > 0.0) {
      const double inv = rsqrt(W + wj);
      c = sqrt(wj) * inv;
      s = sqrt(W) * inv;
    }
    ++m;
    rot_sym(c, s, a, b, 0);
    double bulge = 0.0;
    if (m > 2) {
      bulge = s * b[1];
      b[1] *= c;
    }
    for (int kk = 1; kk < m - 1 && bulge != 0.0; ++kk) {
      double rr;
      givens(b[kk - 1], bulge, c, s, rr);
      b[kk - 1] = rr;
      rot_sym(c, s, a, b, kk);
      if (kk + 1 < m - 1) {
        bulge = s * b[kk + 1];
        b[kk + 1] *= c;
      } else {
        bulge = 0.0;
      }
    }
    W += wj;
  }
  return W;
}

// Work rows (d, e, u and the Jacobi diagonal a) live in shared memory when
// they fit: the rotation chains read values the same thread just wrote, and
// through global memory each of those round trips costs an L2 latency.
constexpr int SPEC_THREADS = 4;
constexpr size_t SPEC_SMEM_MAX = 96 * 1024;

template <bool SMEM>
__global__ void k_spectral(const double *__restrict__ alpha, const double *__restrict__ beta,
                           const double *__restrict__ beta0, const int *__restrict__ k_eff, int B,
                           int k, double *sd, double *se, double *su, JacobiBufs jb,
                           unsigned long long *min_theta_bits, unsigned *status) {
  extern __shared__ double sm[];
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= B) return;
  const int n = k_eff[v];
  jb.n[v] = n;
  if (n <= 0) {
    jb.w0[v] = 0.0;
    return;
  }
  double *d, *e, *u, *a;
  if (SMEM) {
    double *base = sm + (size_t)threadIdx.x * 4 * k;
    d = base;
    e = base + k;
    u = base + 2 * k;
    a = base + 3 * k;
  } else {
    d = sd + (size_t)v * k;
    e = se + (size_t)v * k;
    u = su + (size_t)v * k;
    a = jb.a + (size_t)v * k;
  }
  for (int i = 0; i < n; ++i) {
    d[i] = alpha[(size_t)v * k + i];
    e[i] = (i + 1 < n) ? beta[(size_t)v * k + i] : 0.0;
  }
  if (!tridiag_eig_first_row(d, e, u, n)) {
    atomicOr(status, ST_NO_CONV);
    jb.n[v] = 0;
    jb.w0[v] = 0.0;
    return;
  }
  const double b0 = beta0[v];
  double tmin = d[0];
  // Gauss nodes -> (Omega_j, wt_j) in place: d <- Omega, u <- wt
  for (int i = 0; i < n; ++i) {
    const double th = d[i];
    tmin = fmin(tmin, th);
    const double Om = th > 0.0 ? sqrt(th) : 0.0;
    d[i] = Om;
    u[i] = (Om > 0.0) ? b0 * b0 * u[i] * u[i] / Om : 0.0;
  }
  if (!(tmin > 0.0)) {
    atomicOr(status, ST_NOT_SPD);
  } else {
    atomicMin(min_theta_bits, (unsigned long long)__double_as_longlong(tmin));
  }
  const double W = jacobi_from_nodes(d, u, n, a, e);
  double *ga = jb.a + (size_t)v * k, *b2 = jb.b2 + (size_t)v * k;
  for (int i = 0; i < n; ++i) {
    if (SMEM) ga[i] = a[i];
    b2[i] = (i + 1 < n) ? e[i] * e[i] : 0.0;
  }
  jb.w0[v] = W;
}

void launch_spectral_impl(const double *alpha, const double *beta, const double *beta0,
                          const int *k_eff, int B, int k, JacobiBufs jb, double *scratch,
                          unsigned long long *min_theta_bits, unsigned *status, cudaStream_t st) {
  const int th = SPEC_THREADS;
  const size_t smem = (size_t)th * 4 * k * sizeof(double);
  const dim3 grid((B + th - 1) / th);
  if (smem <= SPEC_SMEM_MAX) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_spectral<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)SPEC_SMEM_MAX);
      attr = true;
    }
    k_spectral<true><<<grid, th, smem, st>>>(alpha, beta, beta0, k_eff, B, k, nullptr, nullptr,
                                             nullptr, jb, min_theta_bits, status);
  } else {
    k_spectral<false><<<grid, th, 0, st>>>(alpha, beta, beta0, k_eff, B, k, scratch,
                                           scratch + (size_t)B * k, scratch + (size_t)2 * B * k,
                                           jb, min_theta_bits, status);
  }
}
}  // namespace lgw
