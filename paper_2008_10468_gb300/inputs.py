"""Seeded synthetic particle populations and sweep points.

This module is the only thing the CUDA path and the CPU oracle share: it
draws workload inputs (momenta, per-particle fields, types, ids) and holds
none of the event generator's arithmetic.  The recipes stand in for the
laser-plasma cascade workloads of the paper (Sec. 3.1.2), whose datasets are
not public; every draw is from numpy's seeded PCG64 generator.

Field geometry.  In the particle populations every particle meets a local
crossed field head-on, as an electron beam meets a laser pulse: with n = p/|p|
and a random unit vector e1 perpendicular to n, E = E0 e1 and
B = -E0 (n x e1), so eps*E + p x B = (eps + |p|) E0 e1 and p.E = 0.  The
quantum parameter is then (eps + |p|) E0 / E_s, and the amplitude E0 is set
from the target value with this closed form.  Recoil lowers |p| and with it
chi, so no particle runs away; amplitudes stay within a few times 10^4
m c omega / e.  In the cascade batch every cell has one crossed field
E = E0 y^, B = E0 z^ and isotropic particles, where the same closed form reads
chi = E0 (eps - p_x) / E_s.
"""
import numpy as np

# Schwinger field in units of m c omega / e for lambda = 1 um:
# m c^2 / (hbar omega) with CODATA 2022 constants.
_HBAR_C_EV_M = 1.973269804e-7        # hbar c in eV m
_MC2_EV = 0.51099895069e6            # m c^2 in eV


def schwinger_field_code_units(lambda_m=1e-6):
    hbar_omega = 2.0 * np.pi * _HBAR_C_EV_M / lambda_m
    return _MC2_EV / hbar_omega


E_S = schwinger_field_code_units()

TYPE_ELECTRON, TYPE_POSITRON, TYPE_PHOTON, TYPE_REMOVED = 0, 1, 2, 3
FIELDS = ("px", "py", "pz", "Ex", "Ey", "Ez", "Bx", "By", "Bz", "w")


def _loguniform(rng, lo, hi, n):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))


def _isotropic(rng, n):
    mu = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    return mu, s * np.cos(phi), s * np.sin(phi)


def _head_on_fields(rng, p, eps, chi_target):
    """E, B (n,3) of a crossed field met head-on by momentum p with target chi."""
    n = p / np.linalg.norm(p, axis=1, keepdims=True)
    # a unit vector perpendicular to n, at a random angle around n
    a = np.where(np.abs(n[:, :1]) < 0.9, [[1.0, 0.0, 0.0]], [[0.0, 1.0, 0.0]])
    u = np.cross(a, n)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = np.cross(n, u)
    phi = rng.uniform(0.0, 2.0 * np.pi, len(p))[:, None]
    e1 = np.cos(phi) * u + np.sin(phi) * v
    E0 = chi_target * E_S / (eps + np.linalg.norm(p, axis=1))
    E = E0[:, None] * e1
    B = -E0[:, None] * np.cross(n, e1)
    return E, B


def _assemble(p, E, B, types, ids, weight=None):
    n = p.shape[0]
    f32 = np.float32
    out = {
        "px": p[:, 0].astype(f32), "py": p[:, 1].astype(f32), "pz": p[:, 2].astype(f32),
        "Ex": E[:, 0].astype(f32), "Ey": E[:, 1].astype(f32), "Ez": E[:, 2].astype(f32),
        "Bx": B[:, 0].astype(f32), "By": B[:, 1].astype(f32), "Bz": B[:, 2].astype(f32),
        "w": np.ones(n, f32) if weight is None else weight.astype(f32),
        "id": ids.astype(np.uint64), "type": types.astype(np.uint8),
    }
    return out


def uniform_field_electrons(n, seed, gamma=(1e2, 1e4), chi=(0.1, 10.0), ptype=TYPE_ELECTRON):
    """Static crossed field (|E| = |B|, B perpendicular to E) met head-on;
    gamma and chi log-uniform, isotropic directions.

    Default ranges: gamma in [1e2, 1e4], chi in [0.1, 10]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = _loguniform(rng, gamma[0], gamma[1], n)
    c = _loguniform(rng, chi[0], chi[1], n)
    mu, sy, sz = _isotropic(rng, n)
    pm = np.sqrt(g * g - 1.0)
    p = np.stack([pm * mu, pm * sy, pm * sz], axis=1)
    # fields from the binary32 momenta so that chi is close to its target
    p32 = p.astype(np.float32).astype(np.float64)
    eps = np.sqrt(1.0 + np.sum(p32 * p32, axis=1))
    E, B = _head_on_fields(rng, p32, eps, c)
    types = np.full(n, ptype, dtype=np.uint8)
    return _assemble(p32, E, B, types, np.arange(n, dtype=np.uint64))


def clumped_mixed(n, seed, hot_fraction=0.01, hot_chi=(10.0, 100.0), hot_gamma=(3e3, 3e4),
                  cold_chi=(1e-3, 1e-2), cold_gamma=(1e2, 1e3)):
    """Mixed population: 25% e-, 25% e+, 50% photons in random order; a contiguous
    block of `hot_fraction` of the indices (the clump) has large chi."""
    rng = np.random.Generator(np.random.PCG64(seed))
    types = np.empty(n, dtype=np.uint8)
    q = n // 4
    types[:q] = TYPE_ELECTRON
    types[q:2 * q] = TYPE_POSITRON
    types[2 * q:] = TYPE_PHOTON
    rng.shuffle(types)
    n_hot = int(round(n * hot_fraction))
    h0 = (n - n_hot) // 2
    hot = np.zeros(n, dtype=bool)
    hot[h0:h0 + n_hot] = True
    g = np.where(hot, _loguniform(rng, hot_gamma[0], hot_gamma[1], n),
                 _loguniform(rng, cold_gamma[0], cold_gamma[1], n))
    c = np.where(hot, _loguniform(rng, hot_chi[0], hot_chi[1], n),
                 _loguniform(rng, cold_chi[0], cold_chi[1], n))
    mu, sy, sz = _isotropic(rng, n)
    photon = types == TYPE_PHOTON
    pm = np.where(photon, g, np.sqrt(g * g - 1.0))
    p = np.stack([pm * mu, pm * sy, pm * sz], axis=1)
    p32 = p.astype(np.float32).astype(np.float64)
    p2 = np.sum(p32 * p32, axis=1)
    eps = np.where(photon, np.sqrt(p2), np.sqrt(1.0 + p2))
    E, B = _head_on_fields(rng, p32, eps, c)
    return _assemble(p32, E, B, types, np.arange(n, dtype=np.uint64))


def cascade_cells(n_cells, seed, n_min=1, n_max=65536, exponent=-1.5,
                  chi_cell=(1e-2, 50.0), gamma=(1e2, 1e4), gamma_ref=1e3):
    """Independent cells with power-law particle counts p(n) ~ n^exponent on
    [n_min, n_max]; each cell has one crossed field whose amplitude gives a
    particle of energy gamma_ref moving along -x the cell value chi_cell/2
    (chi_cell log-uniform).  Electrons, gamma log-uniform, isotropic.

    Returns (arrays, cell_of_particle)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = exponent + 1.0
    u = rng.uniform(0.0, 1.0, n_cells)
    lo, hi = float(n_min) ** a, float(n_max) ** a
    counts = np.floor((lo + u * (hi - lo)) ** (1.0 / a)).astype(np.int64)
    counts = np.clip(counts, n_min, n_max)
    chi_c = _loguniform(rng, chi_cell[0], chi_cell[1], n_cells)
    A = chi_c * E_S / (2.0 * gamma_ref)
    cell = np.repeat(np.arange(n_cells), counts)
    n = int(counts.sum())
    g = _loguniform(rng, gamma[0], gamma[1], n)
    mu, sy, sz = _isotropic(rng, n)
    pm = np.sqrt(g * g - 1.0)
    p = np.stack([pm * mu, pm * sy, pm * sz], axis=1).astype(np.float32).astype(np.float64)
    E0 = A[cell]
    zero = np.zeros(n)
    E = np.stack([zero, E0, zero], axis=1)
    B = np.stack([zero, zero, E0], axis=1)
    types = np.full(n, TYPE_ELECTRON, dtype=np.uint8)
    return _assemble(p, E, B, types, np.arange(n, dtype=np.uint64)), cell


def sweep_points(n, seed, lo=1e-4, hi=50.0):
    """Synchrotron-function arguments, log-uniform in [lo, hi], binary32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(0.0, 1.0, n)
    y = lo * (hi / lo) ** u
    return np.clip(y.astype(np.float32), np.float32(lo), np.float32(hi))


def subset(arrs, idx):
    """Rows `idx` of a particle dict (ids kept)."""
    return {k: np.ascontiguousarray(v[idx]) for k, v in arrs.items()}
