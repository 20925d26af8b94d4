"""Seeded synthetic inputs for the Lanczos GW hot path.

This module only draws random numbers and lays them out; it performs none of
the method's arithmetic (no pair energies, no coupling vectors, no matrix
products).  Both the CPU oracle and the CUDA library consume what it returns.

The paper's workloads (hydrogen-passivated Si clusters, Table 1) are not
available, so seeded stand-ins reproduce their shape: N_c/N_v ~ 8,
N_aux a few times N_v + N_c, Kohn-Sham energies split by a gap, and a
positive semi-definite low-rank Coulomb kernel K = L L^T (Eq. 15-17 give
the density-fitting origin of such factors).

Recipe (numpy PCG64, ``default_rng(seed)``), draws in this order:
  1. eps_v ~ U[-12, -5] eV (n_v values, sorted ascending)
  2. eps_c ~ U[-3, 20] eV  (n_c values, sorted ascending)
  3. L[vc, mu] ~ N(0, sigma_L^2), vc = v * n_c + c   (pair index, v-major)
  4. one coupling factor M in R^{n_aux} per unordered orbital pair
     {t, m}, M ~ N(0, sigma_M^2), drawn in lexicographic order of
     (min(t,m), max(t,m)); (t,m) and (m,t) share it because real orbitals
     make (nm|vc) symmetric in n, m (Eq. 2-3).
sigma_L = 0.05 and sigma_M = 0.1, both divided by sqrt(n_aux) for the
scaled (mid-size and larger) workloads.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    """One synthetic system plus the self-energy request made on it."""

    name: str
    n_v: int
    n_c: int
    n_aux: int
    eps: np.ndarray            # [n_v + n_c] eV, valence block then conduction block
    L: np.ndarray              # [n_v*n_c, n_aux] float64, row vc = v*n_c + c
    targets: np.ndarray        # [n_t] int32 orbital indices (diagonal Sigma_tt)
    m_idx: np.ndarray          # [n_m] int32 summed orbital indices
    M: np.ndarray              # [n_t, n_m, n_aux] float64 coupling factors
    omega: np.ndarray          # [n_freq] eV
    delta: float = 0.05        # broadening (the paper's positive infinitesimal)
    kernel_factor: float = 4.0
    k: int = 64                # Lanczos steps
    meta: dict = field(default_factory=dict)

    @property
    def n_vc(self) -> int:
        return self.n_v * self.n_c

    @property
    def n_t(self) -> int:
        return int(self.targets.shape[0])

    @property
    def n_m(self) -> int:
        return int(self.m_idx.shape[0])


def _pair_factors(rng, targets, m_idx, n_aux, sigma_M):
    pairs = sorted({(min(int(t), int(m)), max(int(t), int(m)))
                    for t in targets for m in m_idx})
    table = {}
    for p in pairs:
        table[p] = rng.normal(0.0, sigma_M, n_aux)
    M = np.empty((len(targets), len(m_idx), n_aux), dtype=np.float64)
    for i, t in enumerate(targets):
        for j, m in enumerate(m_idx):
            M[i, j] = table[(min(int(t), int(m)), max(int(t), int(m)))]
    return M


def make_workload(name, n_v, n_c, n_aux, targets, m_idx, n_freq, seed, *,
                  k=64, omega_lo=-30.0, omega_hi=30.0, delta=0.05,
                  aux_scaled=False, sigma_L=0.05, sigma_M=0.1,
                  kernel_factor=4.0, L_dtype=np.float64):
    rng = np.random.default_rng(seed)
    eps_v = np.sort(rng.uniform(-12.0, -5.0, n_v))
    eps_c = np.sort(rng.uniform(-3.0, 20.0, n_c))
    eps = np.concatenate([eps_v, eps_c]).astype(np.float64)
    s = 1.0 / np.sqrt(n_aux) if aux_scaled else 1.0
    L = rng.standard_normal((n_v * n_c, n_aux), dtype=np.float64)
    L *= sigma_L * s
    if L_dtype is not np.float64:
        L = L.astype(L_dtype)
    targets = np.asarray(targets, dtype=np.int32)
    m_idx = np.asarray(m_idx, dtype=np.int32)
    M = _pair_factors(rng, targets, m_idx, n_aux, sigma_M * s)
    omega = np.linspace(omega_lo, omega_hi, n_freq) if n_freq > 0 else np.zeros(0)
    return Workload(name=name, n_v=n_v, n_c=n_c, n_aux=n_aux, eps=eps, L=L,
                    targets=targets, m_idx=m_idx, M=M, omega=omega,
                    delta=delta, kernel_factor=kernel_factor, k=k,
                    meta=dict(seed=seed, aux_scaled=aux_scaled))


def tiny(seed=0, k=64):
    """Plain-FP64 parity workload: N_v=8, N_c=32 (N_vc=256), N_aux=128,
    targets HOMO-1..LUMO+1 (orbitals 6..9), all 40 orbitals summed,
    200 frequencies on [-30, 30] eV, delta 0.05 eV."""
    n_v, n_c = 8, 32
    return make_workload("tiny", n_v, n_c, 128, list(range(n_v - 2, n_v + 2)),
                         list(range(n_v + n_c)), 200, seed, k=k)


def mid(seed=1, n_targets=32, k=200, n_freq=1000, target_offset=0):
    """Mid-size system: N_v=128, N_c=1024 (N_vc=131072), N_aux=2048, scaled
    distributions.  Targets are HOMO-15..LUMO+15 (32 states); each target
    sums over 256 orbitals (128 valence + lowest 128 conduction).
    ``n_targets``/``target_offset`` select a contiguous slice of the 32."""
    n_v, n_c, A = 128, 1024, 2048
    all_t = list(range(n_v - 16, n_v + 16))
    t = all_t[target_offset:target_offset + n_targets]
    return make_workload("mid", n_v, n_c, A, t, list(range(256)), n_freq, seed,
                         k=k, aux_scaled=True)


def differentiation(seed=4, n_targets=8, n_m=128, k=120, n_freq=1000, target_offset=0):
    """Differentiation workload: N_v=64, N_c=512 (N_vc=32768), N_aux=1024,
    scaled distributions; 8 targets HOMO-3..LUMO+3, each summing over 128
    orbitals (64 valence + lowest 64 conduction); k=120.
    ``n_targets``/``n_m``/``target_offset`` select a subsample."""
    n_v, n_c, A = 64, 512, 1024
    all_t = list(range(n_v - 4, n_v + 4))
    t = all_t[target_offset:target_offset + n_targets]
    return make_workload("differentiation", n_v, n_c, A, t, list(range(n_m)), n_freq, seed,
                         k=k, aux_scaled=True)


def batched_uneven(i, k=150, n_freq=1000, max_targets=None, max_m=256):
    """System i (0..15) of the batched-uneven workload, seed 100+i.  From a
    generator seeded 100+i the shapes are drawn first: N_vc log-uniform in
    [4096, 65536], N_v = max(8, round(sqrt(N_vc / 8))), N_c = round(N_vc /
    N_v), N_aux log-uniform in [512, 2048] rounded to a multiple of 64, and
    the number of targets uniform in {8..64} (straddling the gap).  The
    summed orbitals are all valence states plus the lowest conduction states,
    max_m in total.  Energies, L and M then come from make_workload with the
    same seed and the 1/sqrt(N_aux)-scaled distributions."""
    rng = np.random.default_rng(100 + i)
    n_vc = int(round(np.exp(rng.uniform(np.log(4096), np.log(65536)))))
    n_v = max(8, int(round(np.sqrt(n_vc / 8))))
    n_c = max(1, int(round(n_vc / n_v)))
    A = int(round(np.exp(rng.uniform(np.log(512), np.log(2048))) / 64)) * 64
    n_t = int(rng.integers(8, 65))
    if max_targets is not None:
        n_t = min(n_t, max_targets)
    t0 = max(0, n_v - n_t // 2)
    targets = list(range(t0, min(t0 + n_t, n_v + n_c)))
    m_idx = list(range(min(max_m, n_v + n_c)))
    return make_workload(f"batched{i}", n_v, n_c, A, targets, m_idx, n_freq, 100 + i, k=k,
                         aux_scaled=True)


def large_cluster(n_targets=16, n_m=1024, k=300, n_freq=2000, target_offset=0, seed=5):
    """Large cluster-sized system: N_v=400, N_c=4000 (N_vc=1.6M), N_aux=8192,
    scaled distributions; targets HOMO-7..LUMO+7 (16 states), each summing
    over 1024 orbitals (400 valence + lowest 624 conduction); k=300, 2000
    frequencies.  Returns (workload without L, sigma_L): the 1.6M x 8192
    FP64 factor (105 GB) is drawn by the caller on the device, N(0, sigma_L^2)
    i.i.d. like every other workload here; eps and M follow make_workload's
    recipe (eps from the seeded generator, then M, with no L draws between)."""
    n_v, n_c, A = 400, 4000, 8192
    all_t = list(range(n_v - 8, n_v + 8))
    targets = np.asarray(all_t[target_offset:target_offset + n_targets], dtype=np.int32)
    m_idx = np.asarray(list(range(n_m)), dtype=np.int32)
    rng = np.random.default_rng(seed)
    eps_v = np.sort(rng.uniform(-12.0, -5.0, n_v))
    eps_c = np.sort(rng.uniform(-3.0, 20.0, n_c))
    eps = np.concatenate([eps_v, eps_c]).astype(np.float64)
    s = 1.0 / np.sqrt(A)
    M = _pair_factors(rng, targets, m_idx, A, 0.1 * s)
    omega = np.linspace(-30.0, 30.0, n_freq)
    wl = Workload(name="large_cluster", n_v=n_v, n_c=n_c, n_aux=A, eps=eps, L=None,
                  targets=targets, m_idx=m_idx, M=M, omega=omega, delta=0.05,
                  kernel_factor=4.0, k=k, meta=dict(seed=seed, aux_scaled=True))
    return wl, 0.05 * s


def custom(n_v, n_c, n_aux, n_targets, n_m, n_freq, seed, k, aux_scaled=True):
    """Arbitrary shape with the same recipe: targets straddle the gap,
    the summed set is the lowest ``n_m`` orbitals."""
    lo = max(0, n_v - n_targets // 2)
    t = list(range(lo, min(n_v + n_c, lo + n_targets)))
    return make_workload("custom", n_v, n_c, n_aux, t, list(range(min(n_m, n_v + n_c))),
                         n_freq, seed, k=k, aux_scaled=aux_scaled)
