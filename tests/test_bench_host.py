"""Host-side logic of bench.py (no GPU): the algorithmic work counts behind the roofline,
the recorded-traffic lookup and its source hash, the measured HBM peak."""
import os
import shutil

import pytest

import bench
from paper_1305_4650_gb300 import workloads as wl


def test_phase_ops_follow_the_formulas():
    # part of coordinate 0, the shared parts of the other coordinates (per q phases), the sum of
    # parts, the final step and the 18-op sincos
    assert bench.phase_ops("genradon", 2, 5) == pytest.approx(9 + 9 / 5 + 8 + 12 + 18)
    assert bench.phase_ops("genradon", 3, 4) == pytest.approx(9 + 2 * 9 / 4 + 8 + 12 + 18)
    assert bench.phase_ops("dot", 2, 5) == pytest.approx(5 + 5 / 5 + 1 + 0 + 18)
    assert bench.phase_ops("hypradon", 2, 5) == pytest.approx(4 + 4 / 5 + 8 + 12 + 18)
    # the Fourier phase is the cheapest, the generalized Radon phase the dearest
    ops = {k: bench.phase_ops(k, 2, 5) for k in ("dot", "genradon", "hypradon", "separable")}
    assert min(ops, key=ops.get) == "dot" and max(ops, key=ops.get) == "genradon"


def test_pass_work_counts_match_the_method():
    # d = 2, q = 5, N = 1024: per pair and level (2^d + 1) r phases, (2^{d+1} - 2) q^{d+1} MACs;
    # r^2 phases per pair at the switch; the corner grid point has one non-zero Lagrange node
    spec = wl.genradon2d()
    P, r, q = spec.npts, spec.r, spec.q
    col = bench.pass_work(spec, dict(kind="col", k=3, init=False, switch=True, final=False))
    assert col["phases"] == 3 * 125 * P + r * r * P
    assert col["macs"] == 3 * 6 * q ** 3 * P
    assert col["cmuls"] == 3 * 125 * P and col["cmacs"] == r * r * P
    init = bench.pass_work(spec, dict(kind="col", k=2, init=True, switch=False, final=False))
    assert init["phases"] == 2 * 125 * P + 2 * P
    # the whole default schedule: 10 merge levels, the switch, init and final
    sched = [dict(kind="col", k=2, init=True, switch=False, final=False),
             dict(kind="col", k=3, init=False, switch=True, final=False),
             dict(kind="row", k=2, init=False, switch=False, final=False),
             dict(kind="row", k=3, init=False, switch=False, final=True)]
    total = sum(bench.pass_work(spec, ps)["phases"] for ps in sched)
    assert total == 10 * 125 * P + r * r * P + 4 * P      # 1.97 G phases
    # right-hand sides multiply the arithmetic, not the phases
    w16 = bench.pass_work(spec, sched[1], nrhs=16)
    assert w16["phases"] == col["phases"] and w16["macs"] == 16 * col["macs"]


def test_recorded_traffic_needs_the_recorded_schedule_and_code():
    rec = bench.TRAFFIC["genradon2d"]
    if rec["src_sha256"] != bench.kernel_src_sha256():
        pytest.skip("kernels changed since the traffic was recorded")
    sched = rec["schedule"]
    for i, b in enumerate(rec["bytes"]):
        assert bench.recorded_traffic("genradon2d", sched, i) == b
    assert bench.recorded_traffic("genradon2d", list(reversed(sched)), 1) is None
    assert bench.recorded_traffic("genradon3d", sched, 1) is None
    assert bench.recorded_traffic("genradon2d", sched, len(sched)) is None


def test_source_hash_ignores_comments_not_code(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_1305_4650_gb300", "csrc")
    dst = tmp_path / "paper_1305_4650_gb300" / "csrc"
    dst.mkdir(parents=True)
    for name in bench.TRAFFIC_SRC:
        shutil.copy(os.path.join(src, name), dst / name)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_src_sha256()
    f = dst / bench.TRAFFIC_SRC[0]
    text = f.read_text()
    f.write_text("// a new comment line\n" + text.replace("\n", "\n/* block */\n", 1) + "\n\n")
    assert bench.kernel_src_sha256() == h0
    f.write_text(text.replace("PM_TABLE = 2", "PM_TABLE = 3", 1))
    assert bench.kernel_src_sha256() != h0


def test_measured_hbm_peak_comes_from_the_pool_file():
    gbs, basis = bench.measured_hbm_gbs()
    assert gbs > 1000.0
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert basis.startswith("measured")


@pytest.mark.parametrize("q,kind,off", [(5, 0, 0.0), (5, 0, 0.3), (4, 1, 0.0), (2, 0, 0.0), (3, 0, 0.5), (8, 1, 0.25)])
def test_nonzero_lagrange_count_matches_the_oracle_basis(q, kind, off):
    # the bench's count of non-zero Lagrange values of a grid point (it derives it from the
    # node formula) against the oracle's basis evaluated at that point
    import oracle
    z = oracle.cheb_nodes(q, kind)
    want = sum(1 for t in range(q) if oracle.lagrange1(z, t, off - 0.5) != 0.0)
    assert bench.nonzero_lagrange(q, kind, off - 0.5) == want
