// Continued fractions on the frequency grid (Eq. 14, 10) and the
// quasiparticle equation, FP64.
//
// For a target t and summed orbital m with Jacobi matrix (a, b^2) and total
// weight W of the Omega-space measure (built by the spectral map):
//   Sigma_tm(omega) = -eta_m G(zeta),  zeta = -eta_m (omega - eps_m) + i delta,
//   G(zeta) = W / (zeta - a_0 - b_1^2 / (zeta - a_1 - b_2^2 / (...)))
// which is Eq. 11 (z_m = omega - eps_m - i eta_m delta, zeta = -eta_m z_m).
// Sigma_t = sum over the summed set of Sigma_tm (Eq. 10).
#include <algorithm>

#include "lgw_internal.cuh"

namespace lgw {

struct cplx {
  double re, im;
};

// G(zeta) by bottom-up evaluation of the continued fraction; optionally the
// derivative dG/dzeta by differentiating the recurrence.
template <bool DERIV>
__device__ __forceinline__ void cf_eval(const double *__restrict__ a, const double *__restrict__ b2,
                                        int n, double W, double zr, double zi, cplx &G, cplx &dG) {
  double tr = zr - a[n - 1], ti = zi;
  double dr = 1.0, di = 0.0;   // dT/dzeta
  for (int i = n - 2; i >= 0; --i) {
    const double inv = 1.0 / fma(tr, tr, ti * ti);
    const double q = b2[i] * inv;          // b^2 / T = q * conj(T)
    const double fr = q * tr, fi = -q * ti;
    if (DERIV) {
      // d(b^2/T) = -b^2 dT / T^2 ; T^-2 = conj(T)^2 inv^2
      const double ir = (tr * tr - ti * ti) * inv * inv, ii = -2.0 * tr * ti * inv * inv;
      const double pr = dr * ir - di * ii, pi = dr * ii + di * ir;
      dr = 1.0 + b2[i] * pr;
      di = b2[i] * pi;
    }
    tr = zr - a[i] - fr;
    ti = zi - fi;
  }
  const double inv = 1.0 / fma(tr, tr, ti * ti);
  G.re = W * tr * inv;
  G.im = -W * ti * inv;
  if (DERIV) {
    const double ir = (tr * tr - ti * ti) * inv * inv, ii = -2.0 * tr * ti * inv * inv;
    const double pr = dr * ir - di * ii, pi = dr * ii + di * ir;
    dG.re = -W * pr;
    dG.im = -W * pi;
  }
}

// One thread per (target, frequency, slice of the summed set): loops over its
// slice of m and the continued-fraction depth.  Threads of a warp share t and
// m and read the same coefficients (broadcast loads).  With one slice the
// thread writes Sigma_t(omega_f) itself; otherwise its partial sum goes to
// part[slice] and k_cf_reduce adds the slices in a fixed order.
__global__ void k_cf_grid(CfProblem p, JacobiBufs jb, double *__restrict__ out, int mchunk) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const int ti = blockIdx.y, sl = blockIdx.z;
  if (f >= p.n_freq) return;
  const double om = p.omega[f];
  const int mi0 = sl * mchunk, mi1 = min(p.n_m, mi0 + mchunk);
  double sr = 0.0, si = 0.0;
  for (int mi = mi0; mi < mi1; ++mi) {
    const int v = ti * p.n_m + mi;
    const int n = jb.n[v];
    if (n <= 0) continue;
    const int m = p.m_idx[mi];
    const double eta = (m < p.n_v) ? 1.0 : -1.0;
    const double zr = -eta * (om - p.eps[m]);
    cplx G, dG;
    cf_eval<false>(jb.a + (size_t)v * p.k, jb.b2 + (size_t)v * p.k, n, jb.w0[v], zr, p.delta, G,
                   dG);
    if (jb.g0 == nullptr) {
      sr -= eta * G.re;
      si -= eta * G.im;
    } else {
      // (G(zeta) - G(0)) / z,  z = omega - eps_m - i eta delta
      const double xr = om - p.eps[m], xi = -eta * p.delta;
      const double inv = 1.0 / fma(xr, xr, xi * xi);
      const double nr = G.re - jb.g0[v], ni = G.im;
      sr += (nr * xr + ni * xi) * inv;
      si += (ni * xr - nr * xi) * inv;
    }
  }
  const size_t o = (((size_t)sl * p.n_t + ti) * p.n_freq + f) * 2;
  out[o] = sr;
  out[o + 1] = si;
}

__global__ void k_cf_reduce(const double *__restrict__ part, int S, size_t n,
                            double *__restrict__ sigma) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int sl = 0; sl < S; ++sl) s += part[(size_t)sl * n + i];
  sigma[i] = s;
}

// Sigma_t(E) and dSigma_t/domega at one real E; lanes split the summed set,
// fixed-order warp reduction.  dSigma_tm/domega = dG/dzeta (eta^2 = 1).
__device__ void sigma_at(const CfProblem &p, const JacobiBufs &jb, int ti, double E, cplx &S,
                         cplx &dS) {
  const int lane = threadIdx.x & 31;
  double sr = 0.0, si = 0.0, dr = 0.0, di = 0.0;
  for (int mi = lane; mi < p.n_m; mi += 32) {
    const int v = ti * p.n_m + mi;
    const int n = jb.n[v];
    if (n <= 0) continue;
    const int m = p.m_idx[mi];
    const double eta = (m < p.n_v) ? 1.0 : -1.0;
    cplx G, dG;
    cf_eval<true>(jb.a + (size_t)v * p.k, jb.b2 + (size_t)v * p.k, n, jb.w0[v],
                  -eta * (E - p.eps[m]), p.delta, G, dG);
    if (jb.g0 == nullptr) {
      sr -= eta * G.re;
      si -= eta * G.im;
      dr += dG.re;
      di += dG.im;
    } else {
      // S = (G(zeta) - G(0)) / z, zeta = -eta z:
      // dS/dz = -eta G'(zeta) / z - S / z
      const double xr = E - p.eps[m], xi = -eta * p.delta;
      const double inv = 1.0 / fma(xr, xr, xi * xi);
      const double nr = G.re - jb.g0[v], ni = G.im;
      const double qr = (nr * xr + ni * xi) * inv, qi = (ni * xr - nr * xi) * inv;
      sr += qr;
      si += qi;
      const double gr = -eta * dG.re - qr, gi = -eta * dG.im - qi;
      dr += (gr * xr + gi * xi) * inv;
      di += (gi * xr - gr * xi) * inv;
    }
  }
  S.re = warp_sum(sr);
  S.im = warp_sum(si);
  dS.re = warp_sum(dr);
  dS.im = warp_sum(di);
}

// QP equation E = e0 + Re Sigma_t(E), e0 = eps_t + s_t: Newton from e0; if it
// fails, bracket sign changes of f on the grid (from the grid values of
// Sigma), bisect each and keep the root nearest e0 (ties: larger Z).
// One warp per target.
__global__ void k_qp(CfProblem p, JacobiBufs jb, const double *__restrict__ sigma, int max_iter,
                     double tol, double *e_qp, double *z_qp, unsigned *status) {
  const int ti = blockIdx.x;
  const int t = p.targets[ti];
  const double e0 = p.eps[t] + (p.shift ? p.shift[ti] : 0.0);
  double E = e0;
  bool ok = false;
  cplx S, dS;
  if (p.qp_mode == 1) {
    // linearised: E = e0 + Z Re Sigma(e0), Z = 1 / (1 - Re Sigma'(e0))
    sigma_at(p, jb, ti, e0, S, dS);
    const double Z = 1.0 / (1.0 - dS.re);
    if ((threadIdx.x & 31) == 0) {
      e_qp[ti] = e0 + Z * S.re;
      if (z_qp) z_qp[ti] = Z;
    }
    return;
  }
  for (int it = 0; it < max_iter; ++it) {
    sigma_at(p, jb, ti, E, S, dS);
    const double f = E - e0 - S.re;
    const double fp = 1.0 - dS.re;
    const double dE = f / fp;
    if (fp == 0.0 || !isfinite(dE)) break;
    E -= dE;
    if (fabs(dE) <= tol * fmax(1.0, fabs(E))) {
      ok = true;
      break;
    }
  }
  double Z = 0.0;
  if (ok) {
    sigma_at(p, jb, ti, E, S, dS);
    Z = 1.0 / (1.0 - dS.re);
  } else {
    bool found = false;
    double best_r = 0.0, best_z = 0.0, best_d = 0.0;
    const double *sg = sigma + (size_t)ti * p.n_freq * 2;
    for (int g = 0; g + 1 < p.n_freq; ++g) {
      const double f0 = p.omega[g] - e0 - sg[2 * g];
      const double f1 = p.omega[g + 1] - e0 - sg[2 * g + 2];
      if (!(f0 == 0.0 || f0 * f1 < 0.0)) continue;
      double lo = p.omega[g], hi = p.omega[g + 1], flo = f0;
      double mid = 0.5 * (lo + hi);
      for (int it = 0; it < 200; ++it) {
        mid = 0.5 * (lo + hi);
        sigma_at(p, jb, ti, mid, S, dS);
        const double fm = mid - e0 - S.re;
        if ((fm < 0.0) == (flo < 0.0)) {
          lo = mid;
          flo = fm;
        } else {
          hi = mid;
        }
        if (hi - lo <= tol * fmax(1.0, fabs(mid))) break;
      }
      const double r = 0.5 * (lo + hi);
      sigma_at(p, jb, ti, r, S, dS);
      const double zr = 1.0 / (1.0 - dS.re);
      const double dist = fabs(r - e0);
      if (!found || dist < best_d || (dist == best_d && zr > best_z)) {
        found = true;
        best_r = r;
        best_z = zr;
        best_d = dist;
      }
    }
    if (found) {
      E = best_r;
      Z = best_z;
    } else {
      if ((threadIdx.x & 31) == 0) atomicOr(status, ST_NO_CONV);
      E = NAN;
      Z = NAN;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    e_qp[ti] = E;
    if (z_qp) z_qp[ti] = Z;
  }
}

int cf_slices(const CfProblem &p) {
  // enough (target, frequency, slice) threads to hide the FP64 latency of
  // the continued-fraction chains: about 128k, at most 64 slices
  if (p.n_t <= 0 || p.n_freq <= 0 || p.n_m <= 0) return 1;
  const long long tf = (long long)p.n_t * p.n_freq;
  long long S = (131072 + tf - 1) / tf;
  S = std::min<long long>(S, std::min(p.n_m, 64));
  return (int)std::max<long long>(S, 1);
}

int launch_cf_grid(const CfProblem &p, JacobiBufs jb, double *sigma, double *part, int S,
                   cudaStream_t st) {
  if (p.n_freq <= 0 || p.n_t <= 0) return 0;
  if (part == nullptr) S = 1;
  const int mchunk = (p.n_m + S - 1) / S;
  S = std::max(1, (p.n_m + mchunk - 1) / std::max(1, mchunk));
  dim3 grid((p.n_freq + 127) / 128, p.n_t, S);
  k_cf_grid<<<grid, 128, 0, st>>>(p, jb, S == 1 ? sigma : part, std::max(1, mchunk));
  if (S > 1) {
    const size_t n = (size_t)p.n_t * p.n_freq * 2;
    k_cf_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, S, n, sigma);
    return 2;
  }
  return 1;
}

void launch_qp(const CfProblem &p, JacobiBufs jb, const double *sigma, int max_iter, double tol,
               double *e_qp, double *z_qp, unsigned *status, cudaStream_t st) {
  if (p.n_t <= 0) return;
  k_qp<<<p.n_t, 32, 0, st>>>(p, jb, sigma, max_iter, tol, e_qp, z_qp, status);
}

}  // namespace lgw
