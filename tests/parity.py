"""Event-by-event comparison of the CUDA event generator with the oracle.

Protocol:
  * Each particle's events (sub-step index s, kind, child ids) must be
    identical on both sides, up to the particle's first near-tie recorded by
    the oracle: a draw with |y - P| <= oracle.TIE_DRAW * P, or a plan whose
    sub-step count flips inside the relative band of oracle.TIE_PLAN.  From
    that sub-step on the particle (and any child created there or later) is
    exempt.
  * Energy fractions agree to `delta_rtol` (binary32 x^3 against FP64).
  * Particles with no near-tie end in the same state: same type, momentum
    within `p_rtol` of |p|.
"""
from collections import defaultdict, deque

import numpy as np


def _by_parent(ev):
    d = defaultdict(list)
    for e in ev:
        d[int(e["parent_id"])].append(e)
    for k in d:
        d[k].sort(key=lambda e: int(e["s"]))
    return d


def _rows(store):
    return {int(i): r for r, i in enumerate(store["id"])}


def compare(gpu_ev, orc_ev, orc_ties, gpu_store, orc_store, roots, delta_rtol=2e-6,
            p_rtol=2e-5):
    """Return a report dict; report['mismatches'] lists the failures."""
    ties = {}
    for t in orc_ties:
        i = int(t["id"])
        ties[i] = min(ties.get(i, 1 << 62), int(t["s"]))
    g_by = _by_parent(gpu_ev)
    o_by = _by_parent(orc_ev)
    g_rows = _rows(gpu_store)
    o_rows = _rows(orc_store)
    mism = []
    rep = dict(particles=0, exempt=0, events=0, final_checked=0)
    seen = set()
    q = deque(int(r) for r in roots)
    while q:
        pid = q.popleft()
        if pid in seen:
            continue
        seen.add(pid)
        rep["particles"] += 1
        s_tie = ties.get(pid, 1 << 62)
        oe = [e for e in o_by.get(pid, []) if int(e["s"]) < s_tie]
        ge = [e for e in g_by.get(pid, []) if int(e["s"]) < s_tie]
        if len(oe) != len(ge):
            mism.append((pid, "event count", len(ge), len(oe),
                         [int(e["s"]) for e in ge][:8], [int(e["s"]) for e in oe][:8]))
            continue
        ok = True
        for a, b in zip(ge, oe):
            if (int(a["s"]), int(a["kind"]), int(a["child0"]), int(a["child1"])) != \
               (int(b["s"]), int(b["kind"]), int(b["child0"]), int(b["child1"])):
                mism.append((pid, "event", (int(a["s"]), int(a["kind"])),
                             (int(b["s"]), int(b["kind"]))))
                ok = False
                break
            if abs(float(a["delta"]) / float(b["delta"]) - 1.0) > delta_rtol:
                mism.append((pid, "delta", float(a["delta"]), float(b["delta"])))
                ok = False
                break
            rep["events"] += 1
            q.append(int(b["child0"]))
            if int(b["kind"]) == 2:
                q.append(int(b["child1"]))
        if not ok:
            continue
        if s_tie < (1 << 62):
            rep["exempt"] += 1
            continue
        if pid not in g_rows or pid not in o_rows:
            mism.append((pid, "missing row", pid in g_rows, pid in o_rows))
            continue
        rg, ro = g_rows[pid], o_rows[pid]
        if int(gpu_store["type"][rg]) != int(orc_store["type"][ro]):
            mism.append((pid, "type", int(gpu_store["type"][rg]), int(orc_store["type"][ro])))
            continue
        pg = np.array([gpu_store[k][rg] for k in ("px", "py", "pz")], dtype=np.float64)
        po = np.array([orc_store[k][ro] for k in ("px", "py", "pz")], dtype=np.float64)
        scale = max(np.linalg.norm(po), 1e-30)
        if np.max(np.abs(pg - po)) > p_rtol * scale:
            mism.append((pid, "momentum", pg.tolist(), po.tolist()))
            continue
        rep["final_checked"] += 1
    rep["mismatches"] = mism
    return rep
