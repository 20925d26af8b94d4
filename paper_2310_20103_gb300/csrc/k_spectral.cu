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
// One warp per start vector: the Gauss rule of T_k by parallel bisection and
// the product formula for the weights, then the Jacobi rebuild (lane-
// pipelined node insertions); the work rows live in shared memory.
#include <algorithm>

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

// Jacobi matrix (a[0..n), off-diagonal b[0..n-1), not squared) and total
// weight of the discrete measure sum_j wt_j delta(x - x_j), n = number of
// nodes.  Node jn enters as a new leading row with start-vector weight wt_jn:
// one rotation in plane (0, 1) folds it into the start vector, and the bulge
// it leaves in b is chased to the bottom by rotations in planes (kk, kk+1).
//
// The insertions are pipelined over the warp: in each group of 32 nodes,
// lane l inserts node g0 + l and chases its bulge two rows behind lane l-1.
// Rows are stored bottom-up (with m rows present the leading row sits at
// index n - m), so a new leading row shifts nothing.  A rotation in plane
// (kk, kk+1) touches rows kk-1 .. kk+1, so the rotations of one super-step
// are at least three rows apart, and each row that two insertions both
// rotate is rotated by the earlier insertion first: every rotation sees the
// operands it would see in the one-node-at-a-time order.  Wp (n doubles)
// receives the running weights W_jn = sum_{i < jn} wt_i.  All 32 lanes call
// this; the total weight is returned to every lane.
__device__ double jacobi_from_nodes_warp(const double *x, const double *wt, int n, double *a,
                                         double *b, double *Wp) {
  const int lane = threadIdx.x & 31;
  if (n <= 0) return 0.0;
  double Wtot = 0.0;
  if (lane == 0) {
    double W = 0.0;
    for (int j = 0; j < n; ++j) {
      Wp[j] = W;
      W += wt[j];
    }
    Wtot = W;
    a[n - 1] = x[0];
  }
  __syncwarp();
  for (int g0 = 1; g0 < n; g0 += 32) {
    const int nl = min(32, n - g0);
    const bool act = lane < nl;
    const int jn = g0 + lane;
    const int L = n - 1 - jn;   // leading row once node jn is in
    const int m = jn + 1;       // rows after the insertion
    double bulge = 0.0;
    bool live = false;
    // lane l's last chase step (kk = m - 2) comes at super-step 2 l + m - 2
    const int steps = 3 * (nl - 1) + g0;
    for (int tau = 0; tau < steps; ++tau) {
      const int kk = tau - 2 * lane;
      if (act && kk == 0) {
        a[L] = x[jn];
        b[L] = 0.0;
        const double wj = wt[jn], W = Wp[jn];
        double c = 1.0, s = 0.0;
        if (W + wj > 0.0) {
          const double inv = rsqrt(W + wj);
          c = sqrt(wj) * inv;
          s = sqrt(W) * inv;
        }
        rot_sym(c, s, a, b, L);
        bulge = 0.0;
        if (m > 2) {
          bulge = s * b[L + 1];
          b[L + 1] *= c;
        }
        live = bulge != 0.0;
      } else if (act && live && kk >= 1 && kk < m - 1) {
        double c, s, rr;
        givens(b[L + kk - 1], bulge, c, s, rr);
        b[L + kk - 1] = rr;
        rot_sym(c, s, a, b, L + kk);
        if (kk + 1 < m - 1) {
          bulge = s * b[L + kk + 1];
          b[L + kk + 1] *= c;
        } else {
          bulge = 0.0;
        }
        live = bulge != 0.0;
      }
      __syncwarp();
    }
  }
  return __shfl_sync(0xffffffffu, Wtot, 0);
}

// --------------------------------------------------------------------------
// Warp-parallel Gauss rule: one warp per vector, lanes over the eigenvalues.
//   theta_j (the (j+1)-th smallest eigenvalue of T) by bisection on the Sturm
//   count: the number of sign changes of the leading principal minors
//   p_i = det(T_i - x I) is the number of eigenvalues below x (division-free
//   three-term recurrence, rescaled by exact powers of two);
//   u_1j^2 = det(theta_j I - T_2:n) / (d/dtheta det(theta I - T))|theta_j,
//   the product formula prod_i (theta_j - mu_i) / prod_{i != j} (theta_j -
//   theta_i) (mu: eigenvalues of T without its first row and column).
// A lane interleaves up to SPEC_ILP eigenvalues so that their independent
// recurrences hide the FP64 latency.  The Omega-space Jacobi rebuild then
// runs from the nodes and weights in shared memory, its insertions pipelined
// over the lanes.
// --------------------------------------------------------------------------
constexpr int SPEC_ILP = 8;
constexpr double SCALE_UP = 0x1p+500, SCALE_DN = 0x1p-500;
// bit patterns of 2^500 and 2^-500 (biased exponents 1523 and 523)
constexpr unsigned long long kUpBits = 1523ULL << 52, kDnBits = 523ULL << 52;

// sign with the Sturm convention for zeros (a zero takes the opposite sign
// of its predecessor): p < 0, or p == 0 and the predecessor was not
// negative.  Tested on the bit pattern, and |p| against the rescaling
// thresholds likewise (bit patterns of non-negative doubles order like
// their values), so that the bisection's FP64 pipe, on which GB300 runs
// 2 lanes per SM clock, issues only the recurrence's subtract, multiply and
// fused multiply-add; the comparisons go to the integer pipe.
__device__ __forceinline__ bool neg_sturm(double p, bool prev_neg) {
  const long long bits = __double_as_longlong(p);
  return ((bits << 1) == 0) ? !prev_neg : (bits < 0);
}
__device__ __forceinline__ unsigned long long abs_bits(double p) {
  return (unsigned long long)__double_as_longlong(p) & 0x7fffffffffffffffULL;
}

__global__ void k_spectral_warp(const double *__restrict__ alpha, const double *__restrict__ beta,
                                const double *__restrict__ beta0, const int *__restrict__ k_eff,
                                int B, int k, int warps, JacobiBufs jb,
                                unsigned long long *min_theta_bits, unsigned *status) {
  extern __shared__ double sm[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v = blockIdx.x * warps + wid;
  if (v >= B) return;
  double *al = sm + (size_t)wid * 6 * k;   // alpha
  double *b2 = al + k;                     // beta^2 (b2[i] couples i, i+1)
  double *th = b2 + k;                     // nodes (theta, then Omega)
  double *wt = th + k;                     // u_1^2, then the Omega-space weights
  double *ja = wt + k;                     // Jacobi diagonal
  double *jb_ = ja + k;                    // Jacobi off-diagonal
  // A depth outside [0, k] (possible only for caller-supplied tridiagonals)
  // is flagged and the vector skipped: its rows hold at most k entries.
  int n = k_eff[v];
  if (n < 0 || n > k) {
    if (lane == 0) atomicOr(status, ST_BAD_INPUT);
    n = 0;
  }
  if (lane == 0) jb.n[v] = n;
  if (n <= 0) {
    if (lane == 0) jb.w0[v] = 0.0;
    return;
  }
  double glo = 1e300, ghi = -1e300;
  for (int i = lane; i < n; i += 32) {
    const double a = alpha[(size_t)v * k + i];
    const double bl = i > 0 ? fabs(beta[(size_t)v * k + i - 1]) : 0.0;
    const double br = i + 1 < n ? fabs(beta[(size_t)v * k + i]) : 0.0;
    al[i] = a;
    b2[i] = (i + 1 < n) ? br * br : 0.0;
    glo = fmin(glo, a - bl - br);
    ghi = fmax(ghi, a + bl + br);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
  }
  __syncwarp();
  const double width = ghi - glo;
  glo -= 1e-12 * width + 1e-300;
  ghi += 1e-12 * width + 1e-300;

  for (int j0 = 0; j0 < n; j0 += 32 * SPEC_ILP) {
    double lo[SPEC_ILP], hi[SPEC_ILP];
    int idx[SPEC_ILP];
#pragma unroll
    for (int r = 0; r < SPEC_ILP; ++r) {
      idx[r] = j0 + lane + 32 * r;
      lo[r] = glo;
      hi[r] = ghi;
    }
    // bisection: count(lo) <= j < count(hi); 60 halvings reach the rounding
    // level of the Gershgorin width
    for (int it = 0; it < 60; ++it) {
      double x[SPEC_ILP], p0[SPEC_ILP], p1[SPEC_ILP];
      int cnt[SPEC_ILP];
      bool pn[SPEC_ILP];
#pragma unroll
      for (int r = 0; r < SPEC_ILP; ++r) {
        x[r] = 0.5 * (lo[r] + hi[r]);
        p0[r] = 1.0;
        p1[r] = al[0] - x[r];
        pn[r] = neg_sturm(p1[r], false);
        cnt[r] = pn[r] ? 1 : 0;
      }
      for (int i = 1; i < n; ++i) {
        const double a = al[i], bb = b2[i - 1];
#pragma unroll
        for (int r = 0; r < SPEC_ILP; ++r) {
          double p2 = fma(a - x[r], p1[r], -bb * p0[r]);
          const bool ng = neg_sturm(p2, pn[r]);
          cnt[r] += (ng != pn[r]) ? 1 : 0;
          pn[r] = ng;
          p0[r] = p1[r];
          p1[r] = p2;
          if (abs_bits(p2) > kUpBits) {
            p0[r] *= SCALE_DN;
            p1[r] *= SCALE_DN;
          } else if (abs_bits(p2) < kDnBits && abs_bits(p0[r]) < kDnBits) {
            p0[r] *= SCALE_UP;
            p1[r] *= SCALE_UP;
          }
        }
      }
#pragma unroll
      for (int r = 0; r < SPEC_ILP; ++r) {
        if (cnt[r] <= idx[r])
          lo[r] = x[r];
        else
          hi[r] = x[r];
      }
    }
    // weights: u_1j^2 = det(theta I - T_2:n) / d/dtheta det(theta I - T)
#pragma unroll
    for (int r = 0; r < SPEC_ILP; ++r) {
      if (idx[r] >= n) continue;
      const double t = 0.5 * (lo[r] + hi[r]);
      double d0 = 1.0, d1 = t - al[0], q0 = 0.0, q1 = 1.0;   // det and derivative
      int ed = 0;
      for (int i = 1; i < n; ++i) {
        const double c = t - al[i], bb = b2[i - 1];
        const double d2 = fma(c, d1, -bb * d0);
        const double q2 = fma(c, q1, fma(-bb, q0, d1));
        d0 = d1;
        d1 = d2;
        q0 = q1;
        q1 = q2;
        if (fmax(fabs(d1), fabs(q1)) > SCALE_UP) {
          d0 *= SCALE_DN;
          d1 *= SCALE_DN;
          q0 *= SCALE_DN;
          q1 *= SCALE_DN;
          ed += 500;
        } else if (fmax(fmax(fabs(d1), fabs(q1)), fmax(fabs(d0), fabs(q0))) < SCALE_DN) {
          d0 *= SCALE_UP;
          d1 *= SCALE_UP;
          q0 *= SCALE_UP;
          q1 *= SCALE_UP;
          ed -= 500;
        }
      }
      double e0 = 1.0, e1 = n > 1 ? t - al[1] : 1.0;
      int ee = 0;
      for (int i = 2; i < n; ++i) {
        const double e2 = fma(t - al[i], e1, -b2[i - 1] * e0);
        e0 = e1;
        e1 = e2;
        if (fabs(e1) > SCALE_UP) {
          e0 *= SCALE_DN;
          e1 *= SCALE_DN;
          ee += 500;
        } else if (fmax(fabs(e1), fabs(e0)) < SCALE_DN) {
          e0 *= SCALE_UP;
          e1 *= SCALE_UP;
          ee -= 500;
        }
      }
      th[idx[r]] = t;
      wt[idx[r]] = fabs(ldexp(e1 / q1, ee - ed));
    }
  }
  __syncwarp();
  // Gauss nodes -> (Omega_j, wt_j) in place; smallest node for the report
  const double b0 = beta0[v];
  double tmin = 1e300;
  bool bad = false;
  for (int i = lane; i < n; i += 32) {
    const double t = th[i];
    tmin = fmin(tmin, t);
    bad |= !(t > 0.0);
    const double Om = t > 0.0 ? sqrt(t) : 0.0;
    th[i] = Om;
    wt[i] = Om > 0.0 ? b0 * b0 * wt[i] / Om : 0.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
  bad = __any_sync(0xffffffffu, bad);
  __syncwarp();
  if (lane == 0) {
    if (bad)
      atomicOr(status, ST_NOT_SPD);
    else
      atomicMin(min_theta_bits, (unsigned long long)__double_as_longlong(tmin));
  }
  // alpha's rows are free now: the running weights of the rebuild
  const double W = jacobi_from_nodes_warp(th, wt, n, ja, jb_, al);
  if (lane == 0) jb.w0[v] = W;
  __syncwarp();
  double *ga = jb.a + (size_t)v * k, *gb2 = jb.b2 + (size_t)v * k;
  for (int i = lane; i < n; i += 32) {
    ga[i] = ja[i];
    gb2[i] = (i + 1 < n) ? jb_[i] * jb_[i] : 0.0;
  }
}

void launch_spectral_impl(const double *alpha, const double *beta, const double *beta0,
                          const int *k_eff, int B, int k, JacobiBufs jb, double *scratch,
                          unsigned long long *min_theta_bits, unsigned *status, cudaStream_t st) {
  // warp-parallel Gauss rule: 6 k doubles of shared memory per warp
  const size_t per_warp = (size_t)6 * k * sizeof(double);
  const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, (200 * 1024) / per_warp));
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_spectral_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const dim3 grid((B + warps - 1) / warps);
  k_spectral_warp<<<grid, 32 * warps, per_warp * warps, st>>>(alpha, beta, beta0, k_eff, B, k,
                                                              warps, jb, min_theta_bits, status);
  (void)scratch;
}

// ---------------------------------------------------------------------------
// Spectral interval of C for the polynomial form (text after Eq. 12: p_g is
// fitted on the range of C's eigenvalues).
// ---------------------------------------------------------------------------
// Start vector with entries uniform in [-1, 1) from a counter-based hash
// (splitmix64 of seed + index), zero in the padding.
__global__ void k_hash_vector(double *v, int n_vc, int N, unsigned long long seed) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N) return;
  if (e >= n_vc) {
    v[e] = 0.0;
    return;
  }
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(e + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  v[e] = (double)(z >> 11) * 0x1p-52 - 1.0;
}

// Number of eigenvalues of the tridiagonal (a, b) below x (Sturm count by
// the LDL^T pivots, zero pivots nudged off zero).
__device__ int sturm_below(const double *a, const double *b, int n, double x, double pivmin) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < n; ++i) {
    const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
    d = a[i] - x - (i > 0 ? bb / d : 0.0);
    if (fabs(d) < pivmin) d = -pivmin;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// One block: out[0] = min over the pairs of Delta^2 (C = Delta^2 + a positive
// semidefinite term, so no eigenvalue lies below it); out[1] = the largest
// Ritz value of the k-step tridiagonal (a, b) plus the last off-diagonal
// b_k = ||C q_k - ...||, the residual norm that bounds how far the Ritz value
// can lie from an eigenvalue.
__global__ void k_interval(const double *__restrict__ Delta2, int n_vc, const double *a,
                           const double *b, const int *k_eff, double *out) {
  __shared__ double red[256];
  double m = 1e300;
  for (int e = threadIdx.x; e < n_vc; e += blockDim.x) m = fmin(m, Delta2[e]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const int n = *k_eff;
  double hi = 0.0;
  if (n > 0) {
    double glo = 1e300, ghi = -1e300, scale = 0.0;
    for (int i = 0; i < n; ++i) {
      const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < n ? fabs(b[i]) : 0.0);
      glo = fmin(glo, a[i] - r);
      ghi = fmax(ghi, a[i] + r);
      scale = fmax(scale, fabs(a[i]) + r);
    }
    const double pivmin = 1e-300 + 1e-15 * scale * 1e-15;
    double lo = glo, up = ghi;   // the largest eigenvalue lies in (lo, up]
    for (int it = 0; it < 200 && up - lo > 1e-14 * scale; ++it) {
      const double mid = 0.5 * (lo + up);
      if (sturm_below(a, b, n, mid, pivmin) >= n) up = mid; else lo = mid;
    }
    hi = up + (n - 1 < 0 ? 0.0 : fabs(b[n - 1]));
  }
  out[0] = red[0];
  out[1] = hi;
}

void launch_interval(const double *Delta2, int n_vc, int N, const double *a, const double *b,
                     const int *k_eff, double *out, double *vec, unsigned long long seed,
                     bool make_vector, cudaStream_t st) {
  if (make_vector)
    k_hash_vector<<<(N + 255) / 256, 256, 0, st>>>(vec, n_vc, N, seed);
  else
    k_interval<<<1, 256, 0, st>>>(Delta2, n_vc, a, b, k_eff, out);
}
}  // namespace lgw
