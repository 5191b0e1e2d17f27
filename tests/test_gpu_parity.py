"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.  GPU only."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2008_10468_gb300 import inputs as I
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2008_10468_gb300 import qed  # noqa: E402

F_TOL = 4e-6  # relative error of F1/F2 in binary32 over [1e-4, 50]


def _ctx(**kw):
    return qed.Context(**kw)


# --------------------------------------------------------------------------
# Synchrotron functions (Sec. 3.2.1)
# --------------------------------------------------------------------------
def _gpu_F(y, ctx=None):
    ctx = ctx or _ctx()
    yd = torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda()
    F1 = torch.empty_like(yd)
    F2 = torch.empty_like(yd)
    ctx.synchrotron_F1F2(yd, F1, F2)
    return F1.cpu().numpy(), F2.cpu().numpy()


def test_synchrotron_1e6_log_uniform_per_decade():
    y = I.sweep_points(1_000_000, 20081048)
    g1, g2 = _gpu_F(y)
    o1, o2 = O.F1F2(y.astype(np.float64))
    e1 = np.abs(g1 / o1 - 1)
    e2 = np.abs(g2 / o2 - 1)
    dec = np.floor(np.log10(y)).astype(int)
    rows = []
    for d in range(-4, 2):
        m = dec == d
        rows.append((d, float(e1[m].max()), float(e2[m].max())))
    print("max rel err per decade (F1, F2):", rows)
    assert e1.max() <= F_TOL and e2.max() <= F_TOL


def test_synchrotron_edges_and_ragged_sizes():
    ctx = _ctx()
    # special values: 0 and >= 88 give 0; tiny and huge handled
    y = np.array([0.0, 1e-30, 1e-12, 2.0 ** -14, 2.0 ** -14 * 0.999, 0.5, 1.0, 64.0, 87.9,
                  88.0, 1e3], np.float32)
    g1, g2 = _gpu_F(y, ctx)
    o1, o2 = O.F1F2(y.astype(np.float64))
    assert g1[0] == 0.0 and g2[0] == 0.0
    assert g1[-1] == 0.0 and g2[-2] == 0.0
    for i in range(1, 9):
        assert abs(g1[i] / o1[i] - 1) < F_TOL and abs(g2[i] / o2[i] - 1) < F_TOL, (y[i], g1[i], o1[i])
    # ragged lengths and a misaligned base exercise the scalar tail
    base = I.sweep_points(5000, 3)
    o1, o2 = O.F1F2(base.astype(np.float64))
    yd = torch.from_numpy(base).cuda()
    for off, n in ((0, 1), (0, 3), (1, 4097), (3, 997), (0, 0)):
        view = yd[off:off + n]
        F1 = torch.zeros(n + 1, device="cuda")[1:]
        F2 = torch.zeros(n, device="cuda")
        ctx.synchrotron_F1F2(view, F1, F2)
        if n:
            assert np.max(np.abs(F1.cpu().numpy() / o1[off:off + n] - 1)) < F_TOL
            assert np.max(np.abs(F2.cpu().numpy() / o2[off:off + n] - 1)) < F_TOL
    # one output only
    F2 = torch.zeros(5000, device="cuda")
    ctx.synchrotron_F1F2(yd, None, F2)
    assert np.max(np.abs(F2.cpu().numpy() / o2 - 1)) < F_TOL


def test_synchrotron_generated_arguments():
    ctx = _ctx()
    n = 1 << 16
    y = torch.empty(n, device="cuda")
    F1 = torch.empty(n, device="cuda")
    F2 = torch.empty(n, device="cuda")
    chk = torch.zeros(1, device="cuda")
    ctx.synchrotron_generate(1234, n, 1e-4, 50.0, chk, y, F1, F2)
    yh = y.cpu().numpy()
    assert yh.min() >= 1e-4 * (1 - 1e-6) and yh.max() <= 50.0 * (1 + 1e-6)
    # arguments follow the Philox stream: y = lo (hi/lo)^u
    r = O.philox([5, 0, 0, 0], [1234, 0])
    u = O.uniform(r[2])
    assert yh[22] == pytest.approx(1e-4 * (5e5) ** u, rel=2e-6)
    o1, o2 = O.F1F2(yh.astype(np.float64))
    assert np.max(np.abs(F1.cpu().numpy() / o1 - 1)) < F_TOL
    assert np.max(np.abs(F2.cpu().numpy() / o2 - 1)) < F_TOL
    assert float(chk.item()) == pytest.approx(float(np.sum(o1 + o2)), rel=1e-4)


def test_synchrotron_full_sweep_sampled():
    """2^28 points (the sweep workload) through the array path; 1e6 sampled."""
    n = 1 << 28
    y = I.sweep_points(n, 20081048)
    ctx = _ctx()
    yd = torch.from_numpy(y).cuda()
    F1 = torch.empty_like(yd)
    F2 = torch.empty_like(yd)
    ctx.synchrotron_F1F2(yd, F1, F2)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(n, 1_000_000, replace=False))
    ti = torch.from_numpy(idx).cuda()
    g1 = F1[ti].cpu().numpy()
    g2 = F2[ti].cpu().numpy()
    o1, o2 = O.F1F2(y[idx].astype(np.float64))
    assert np.max(np.abs(g1 / o1 - 1)) <= F_TOL
    assert np.max(np.abs(g2 / o2 - 1)) <= F_TOL


# --------------------------------------------------------------------------
# Planner (Algorithms 1/2, planning; Sec. 3.1.1)
# --------------------------------------------------------------------------
def _oracle_plans(cf, arr, rows):
    chi = np.zeros(len(rows))
    N = np.zeros(len(rows), dtype=np.int64)
    tie = np.zeros(len(rows), dtype=bool)
    eps = O.TIE_PLAN
    for j, i in enumerate(rows):
        photon = arr["type"][i] == 2
        p = (arr["px"][i], arr["py"][i], arr["pz"][i])
        E = (arr["Ex"][i], arr["Ey"][i], arr["Ez"][i])
        B = (arr["Bx"][i], arr["By"][i], arr["Bz"][i])
        N[j], chi[j], g, f = O.plan(cf, p, E, B, 0.1, photon=photon)
        # tie: the count changes inside the relative band
        q = f / cf.p_max
        tie[j] = math.ceil(q * (1 - eps)) != math.ceil(q * (1 + eps))
    return chi, N, tie


@pytest.mark.parametrize("workload", ["uniform", "clumped"])
def test_plan_parity(workload):
    if workload == "uniform":
        arr = I.uniform_field_electrons(100_000, 20081047)
        rows = np.arange(0, 100_000, 7)
        mask = 1
    else:
        arr = I.clumped_mixed(1 << 20, 20081049)
        rng = np.random.default_rng(1)
        rows = np.sort(rng.choice(1 << 20, 30_000, replace=False))
        mask = 3
    n = len(arr["px"])
    ctx = _ctx(process_mask=mask)
    store = qed.ParticleStore.from_numpy(arr)
    chi = torch.empty(n, device="cuda")
    N = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.plan(store, n, chi, N)
    gchi = chi.cpu().numpy()[rows]
    gN = N.cpu().numpy().view(np.uint32)[rows].astype(np.int64)
    cf = O.make_config(1, process_mask=mask)
    ochi, oN, tie = _oracle_plans(cf, arr, rows)
    rel = np.abs(gchi / np.maximum(ochi, 1e-300) - 1)
    print("plan: max chi rel err %.2e, ties %d of %d" % (rel.max(), tie.sum(), len(rows)))
    assert rel.max() < 1e-6
    bad = (gN != oN) & ~tie
    assert not bad.any(), list(zip(rows[bad][:5], gN[bad][:5], oN[bad][:5]))


def test_plan_cells_parity():
    """Per-cell counts (one sub-step per cell, Algorithms 1 and 2) against the
    oracle; cells holding a row whose own count is a near-tie are exempt."""
    n = 40_000
    arr = I.clumped_mixed(n, 20081049, hot_fraction=0.02)
    rng = np.random.default_rng(4)
    ncells = 5000
    cell = rng.integers(0, ncells + 50, n).astype(np.uint32)   # ~1% out of range
    ctx = _ctx()
    store = qed.ParticleStore.from_numpy(arr)
    cd = torch.from_numpy(cell.view(np.int32)).cuda()
    g = ctx.plan_cells(store, n, cd, ncells).cpu().numpy().view(np.uint32).astype(np.int64)
    cf = O.make_config(1, process_mask=3)
    o = O.plan_cells(cf, arr, cell, ncells)
    _, _, tie = _oracle_plans(cf, arr, np.arange(n))
    tied_cells = set(cell[tie].tolist())
    ok = np.array([c not in tied_cells for c in range(ncells)])
    print("plan_cells: %d cells, %d exempt, max count %d" % (ncells, (~ok).sum(), o.max()))
    assert (~ok).sum() < 0.01 * ncells
    assert np.array_equal(g[ok], o[ok]), np.nonzero((g != o) & ok)[0][:5]
    # the count of every cell is a multiple-row maximum: check one against qed_plan
    N = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.plan(store, n, None, N)
    Nh = N.cpu().numpy().astype(np.int64)
    c0 = int(cell[0])
    if c0 < ncells:
        assert g[c0] == Nh[cell == c0].max()
    # no rows, no cells
    assert ctx.plan_cells(store, 0, cd, ncells).sum().item() == 0
    ctx.plan_cells(store, n, cd, 0)


def test_plan_cells_grouped_rows():
    """Per-cell counts with the rows of each cell together in the store (a PIC
    code's cell-sorted particles): there the 32 rows of a warp often share one
    cell and fold their counts into a single atomic.  Cells of 1 to 4096 rows
    (power law), a run of removed rows inside a cell, a cell whose indices are
    out of range, and a row count that is not a multiple of 32.  Every count
    equals the maximum of qed_plan's counts over the cell's rows, and the
    oracle's count outside near-ties."""
    arr, cell = I.cascade_cells(400, 20081051, n_max=4096)
    n = len(cell)
    n -= 3 if (n - 3) % 32 else 4
    arr = {k: np.ascontiguousarray(v[:n]) for k, v in arr.items()}
    cell = cell[:n].astype(np.uint32)
    ncells = int(cell.max()) + 1
    big = int(np.argmax(np.bincount(cell)))
    rows_big = np.nonzero(cell == big)[0]
    arr["type"][rows_big[40:100]] = I.TYPE_REMOVED      # removed rows inside a cell
    other = int(cell[rows_big[-1] + 1]) if rows_big[-1] + 1 < n else int(cell[0])
    cell = np.where(cell == other, ncells + 7, cell).astype(np.uint32)   # out of range
    sizes = np.bincount(cell[cell < ncells], minlength=ncells)
    assert sizes.max() >= 64 and (sizes[sizes > 0] < 32).any()
    ctx = _ctx(process_mask=3)
    store = qed.ParticleStore.from_numpy(arr)
    cd = torch.from_numpy(cell.view(np.int32)).cuda()
    g = ctx.plan_cells(store, n, cd, ncells).cpu().numpy().view(np.uint32).astype(np.int64)
    N = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.plan(store, n, None, N)
    Nh = N.cpu().numpy().view(np.uint32).astype(np.int64)
    want = np.zeros(ncells, dtype=np.int64)
    inr = cell < ncells
    np.maximum.at(want, cell[inr].astype(np.int64), Nh[inr])
    assert np.array_equal(g, want), np.nonzero(g != want)[0][:5]
    assert g[other] == 0
    cf = O.make_config(1, process_mask=3)
    o = O.plan_cells(cf, arr, cell, ncells)
    _, _, tie = _oracle_plans(cf, arr, np.arange(n))
    tied = set(cell[tie & inr & (arr["type"] <= 2)].tolist())
    ok = np.array([c not in tied for c in range(ncells)])
    print("plan_cells grouped: %d rows, %d cells (largest %d rows), %d exempt" %
          (n, ncells, sizes.max(), (~ok).sum()))
    assert (~ok).sum() < 0.02 * ncells
    assert np.array_equal(g[ok], o[ok]), np.nonzero((g != o) & ok)[0][:5]


# --------------------------------------------------------------------------
# Event step (Algorithms 1 and 2)
# --------------------------------------------------------------------------
def _run_gpu(arr, step, capacity, log_cap=1 << 20, **cfg):
    ctx = _ctx(**cfg)
    ctx.set_event_log(log_cap)
    store = qed.ParticleStore.from_numpy(arr, capacity=capacity)
    st = ctx.event_step(store, step)
    ev, nev = ctx.read_event_log()
    assert nev <= log_cap
    return store.to_numpy(), st, ev


def _check(arr, step, capacity, seed, mask=3, cascade=True, recoil=True, max_exempt=1e-3):
    g_store, g_st, g_ev = _run_gpu(arr, step, capacity, seed=seed, process_mask=mask,
                                   cascade=cascade, recoil=recoil)
    cf = O.make_config(seed, process_mask=mask, cascade=int(cascade), recoil=int(recoil))
    o_store, o_st, o_ev, o_ties = O.event_step(cf, arr, step, capacity=capacity)
    assert g_st["status"] == 0 and o_st["status"] == 0
    rep = parity.compare(g_ev, o_ev, o_ties, g_store, o_store, arr["id"])
    print("parity:", {k: v for k, v in rep.items() if k != "mismatches"},
          "gpu", g_st, "oracle", o_st)
    assert not rep["mismatches"], rep["mismatches"][:5]
    print("exempt fraction %.2e" % (rep["exempt"] / max(rep["particles"], 1)))
    assert rep["exempt"] <= max_exempt * rep["particles"]
    if len(o_ties) == 0:
        for k in ("substeps", "emissions", "pairs", "children", "plans"):
            assert g_st[k] == o_st[k], k
    return rep, g_st, o_st


def test_event_step_uniform_field_emission():
    # the uniform-field electron workload (gamma 1e2..1e4, chi 0.1..10), 300 rows
    arr = I.uniform_field_electrons(300, 20081047)
    _check(arr, 0, capacity=300 * 200, seed=20081047, mask=1, cascade=False)


def test_event_step_clumped_cascade():
    # mixed e-/e+/photon population with a hot clump; emission + pairs + cascade
    arr = I.clumped_mixed(4133, 20081049, hot_fraction=0.02)
    _check(arr, 3, capacity=4133 * 20, seed=20081049, mask=3, cascade=True)


def test_event_step_without_recoil_validation_mode():
    arr = I.clumped_mixed(1500, 77, hot_fraction=0.05)
    _check(arr, 1, capacity=1500 * 40, seed=77, mask=3, cascade=True, recoil=False)


def test_event_step_pairs_only():
    arr = I.clumped_mixed(2000, 8, hot_fraction=0.1)
    _check(arr, 2, capacity=2000 * 4, seed=8, mask=2, cascade=False)


@pytest.mark.parametrize("n", [1, 2, 31, 33, 64])
def test_tiny_populations_over_several_steps(n):
    # brute force on tiny stores: every particle, every event, three global
    # steps, each started from the GPU's own result (children included)
    arr = I.clumped_mixed(max(n, 4), 500 + n, hot_fraction=0.5)
    arr = {k: v[:n] for k, v in arr.items()}
    for step in range(3):
        g_store, g_st, g_ev = _run_gpu(arr, step, n * 4000, seed=31 + n, process_mask=3,
                                       cascade=True)
        cf = O.make_config(31 + n, process_mask=3, cascade=1)
        o_store, o_st, o_ev, o_ties = O.event_step(cf, arr, step, capacity=n * 4000)
        rep = parity.compare(g_ev, o_ev, o_ties, g_store, o_store, arr["id"])
        assert g_st["status"] == 0 and o_st["status"] == 0
        assert not rep["mismatches"], (step, rep["mismatches"][:3])
        if len(o_ties) == 0:
            for k in ("substeps", "emissions", "pairs", "children", "plans"):
                assert g_st[k] == o_st[k], (step, k)
        arr = g_store


def _crossed_beam(M, gamma, chi_t, photon=False):
    """M identical particles meeting a crossed field head-on (E0 y, B0 z, moving -x)."""
    f32 = np.float32
    pm = gamma if photon else math.sqrt(gamma * gamma - 1.0)
    E0 = np.float32(chi_t * O.schwinger_field() / (gamma + pm))
    arr = {"px": np.full(M, -pm, f32), "py": np.zeros(M, f32), "pz": np.zeros(M, f32),
           "Ex": np.zeros(M, f32), "Ey": np.full(M, E0, f32), "Ez": np.zeros(M, f32),
           "Bx": np.zeros(M, f32), "By": np.zeros(M, f32), "Bz": np.full(M, E0, f32),
           "w": np.ones(M, f32), "id": np.arange(M, dtype=np.uint64),
           "type": np.full(M, 2 if photon else 0, np.uint8)}
    chi, g = O.chi((-pm, 0.0, 0.0), (0.0, float(E0), 0.0), (0.0, 0.0, float(E0)), photon=photon)
    return arr, chi, g


def _x_cdf(kind, b, x):
    """Normalised CDF of the event variable at x from the oracle's acceptance
    function (Gauss-Legendre): x = delta^{1/3} for emission, delta_e for pairs."""
    xs, ws = np.polynomial.legendre.leggauss(24)
    f = O.Pm if kind == 0 else O.Pp

    def integ(a, c, panels):
        edges = np.linspace(a, c, panels + 1)
        tot = 0.0
        for lo, hi in zip(edges[:-1], edges[1:]):
            for xx, ww in zip(0.5 * (lo + hi) + 0.5 * (hi - lo) * xs, ws):
                tot += 0.5 * (hi - lo) * ww * f(b, 1.0, float(xx))
        return tot
    return integ(0.0, x, 12) / integ(0.0, 1.0, 24)


def test_emission_spectrum_ks_against_oracle_and_closed_form():
    # no recoil: every event is an independent draw from the spectrum at fixed
    # (chi, gamma); GPU and oracle run with different seeds
    from scipy import stats
    arr, chi, g = _crossed_beam(20000, 1000.0, 1.0)
    _, g_st, g_ev = _run_gpu(arr, 0, 20000 * 40, seed=101, process_mask=1, cascade=False,
                             recoil=False)
    small = I.subset(arr, np.arange(3000))
    cf = O.make_config(202, process_mask=1, cascade=0, recoil=0)
    _, o_st, o_ev, _ = O.event_step(cf, small, 0, capacity=3000 * 40)
    xg = np.cbrt(g_ev["delta"].astype(np.float64))
    xo = np.cbrt(o_ev["delta"].astype(np.float64))
    assert len(xg) > 20000 and len(xo) > 3000
    p2 = stats.ks_2samp(xg, xo).pvalue
    grid = np.linspace(0.0, 1.0, 161)
    cdf = np.array([_x_cdf(0, 1.5 * chi, v) if v > 0 else 0.0 for v in grid])
    p1 = stats.kstest(xg, lambda v: np.interp(v, grid, cdf)).pvalue
    print("emission spectrum: KS GPU vs oracle p=%.3f, GPU vs closed form p=%.3f" % (p2, p1))
    assert p2 > 0.01 and p1 > 0.01


def test_pair_spectrum_ks_and_symmetry():
    # photons at chi_gamma ~ 5, pairs only, no recoil (the photon is kept, so
    # its decays are independent draws); the electron fraction is symmetric
    # about 1/2
    from scipy import stats
    arr, chi, g = _crossed_beam(20000, 2000.0, 5.0, photon=True)
    _, g_st, g_ev = _run_gpu(arr, 0, 20000 * 40, seed=303, process_mask=2, cascade=False,
                             recoil=False)
    small = I.subset(arr, np.arange(3000))
    cf = O.make_config(404, process_mask=2, cascade=0, recoil=0)
    _, o_st, o_ev, _ = O.event_step(cf, small, 0, capacity=3000 * 40)
    dg = g_ev["delta"].astype(np.float64)
    do = o_ev["delta"].astype(np.float64)
    assert len(dg) > 5000 and len(do) > 500
    p2 = stats.ks_2samp(dg, do).pvalue
    # symmetry about 1/2, on independent data: the distances from 1/2 of the
    # events below and above it have one distribution, and each side holds
    # half of the events (binomial)
    left, right = 0.5 - dg[dg < 0.5], dg[dg > 0.5] - 0.5
    ps = min(stats.ks_2samp(left, right).pvalue,
             stats.binomtest(len(left), len(left) + len(right), 0.5).pvalue)
    grid = np.linspace(0.0, 1.0, 161)
    cdf = np.array([_x_cdf(1, 1.5 * chi, v) if v > 0 else 0.0 for v in grid])
    p1 = stats.kstest(dg, lambda v: np.interp(v, grid, cdf)).pvalue
    print("pair spectrum: KS GPU vs oracle p=%.3f, vs closed form p=%.3f, symmetry p=%.3f"
          % (p2, p1, ps))
    assert p2 > 0.01 and p1 > 0.01 and ps > 0.01


def _sampled_full_size(arr, capacity, seed, mask, roots, log_cap):
    g_store, g_st, g_ev = _run_gpu(arr, 0, capacity, log_cap=log_cap, seed=seed,
                                   process_mask=mask, cascade=True)
    print("full-size step:", g_st)
    assert g_st["status"] == 0
    sub = I.subset(arr, roots)
    cf = O.make_config(seed, process_mask=mask, cascade=1)
    o_store, o_st, o_ev, o_ties = O.event_step(cf, sub, 0, capacity=len(roots) * 4000)
    rep = parity.compare(g_ev, o_ev, o_ties, g_store, o_store, sub["id"])
    print("sampled parity:", {k: v for k, v in rep.items() if k != "mismatches"},
          "exempt fraction %.2e" % (rep["exempt"] / max(rep["particles"], 1)), g_st)
    assert not rep["mismatches"], rep["mismatches"][:5]
    assert rep["exempt"] <= 1e-3 * rep["particles"]
    return g_st


def test_event_step_uniform_field_full_size_sampled():
    arr = I.uniform_field_electrons(100_000, 20081047)
    rng = np.random.default_rng(2)
    roots = np.sort(rng.choice(100_000, 48, replace=False))
    _sampled_full_size(arr, 100_000 * 64, 20081047, 1, roots, 1 << 23)


def test_event_step_clumped_full_size_sampled():
    n = 1 << 24
    arr = I.clumped_mixed(n, 20081049)
    n_hot = int(round(n * 0.01))
    h0 = (n - n_hot) // 2
    rng = np.random.default_rng(3)
    hot = rng.choice(np.arange(h0, h0 + n_hot), 24, replace=False)
    cold = rng.choice(np.concatenate([np.arange(0, h0), np.arange(h0 + n_hot, n)]), 40,
                      replace=False)
    roots = np.sort(np.concatenate([hot, cold]))
    # the hot clump cascades within the step (~85 children per hot particle)
    _sampled_full_size(arr, n + (1 << 25), 20081049, 3, roots, 1 << 25)


# --------------------------------------------------------------------------
# Degenerate inputs and errors
# --------------------------------------------------------------------------
def test_empty_and_removed_and_fieldless():
    ctx = _ctx()
    store = qed.ParticleStore(1024)
    st = ctx.event_step(store, 0)
    assert st["status"] == 0 and st["substeps"] == 0 and st["count"] == 0
    arr = I.clumped_mixed(256, 4)
    arr["type"][:] = 3
    store.load(arr)
    st = ctx.event_step(store, 0)
    assert st["substeps"] == 0 and st["count"] == 256
    arr = I.clumped_mixed(256, 4)
    for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
        arr[k][:] = 0
    store.load(arr)
    st = ctx.event_step(store, 0)
    # no field: chi = 0, one sub-step each, no event
    assert st["emissions"] == 0 and st["pairs"] == 0 and st["substeps"] == 256


def test_capacity_overflow_reports_required_rows():
    arr = I.uniform_field_electrons(2000, 20081047)
    ctx = _ctx(process_mask=1, cascade=False)
    store = qed.ParticleStore.from_numpy(arr, capacity=2100)
    st = ctx.event_step(store, 0)
    assert st["status"] == qed.QED_ERR_CAPACITY
    assert st["required_capacity"] > 2100
    assert store.n() == 2100
    # the context stays usable after the error
    store2 = qed.ParticleStore.from_numpy(I.uniform_field_electrons(100, 1), capacity=100000)
    assert ctx.event_step(store2, 1)["status"] == 0


def test_bad_arguments_are_rejected():
    ctx = _ctx()
    store = qed.ParticleStore(16)
    with pytest.raises(qed.QEDError):
        ctx.event_step(store, 1 << 33)
    with pytest.raises(qed.QEDError):
        qed.Context(p_max=0.0)
