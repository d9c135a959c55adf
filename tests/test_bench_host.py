"""Host-side bookkeeping of bench.py (no GPU): the elementary operations it
counts, the algorithmic flop count of the rounding's R factors, and the TT
against dense error it reports."""
import math

import numpy as np

import bench
import synth
from oracle import pmf, tt


def test_ldu_ops_are_the_oracle_operations():
    for F in (synth.config2().F, synth.config3(d=6, n=16).F,
              np.array([[0.9, 0.3, -0.2], [0.25, 1.1, 0.4], [-0.3, 0.2, 0.8]])):
        ours = bench.ldu_ops(F)
        ref = pmf.elementary_ops(F)
        assert len(ours) == len(ref)
        for a, b in zip(ours, ref):
            assert a[0] == b[0] and a[1:-1] == tuple(b[1:-1])
            assert abs(a[-1] - b[-1]) < 1e-14


def test_shear_spans_and_algorithmic_flops_of_the_bench_workload():
    model = synth.config2(n=128)
    spans = [bench.shear_span(model, m, n, a) for kind, m, n, a in
             (op for op in bench.ldu_ops(model.F) if op[0] == "shear")]
    assert spans == [7, 5, 7, 9, 5, 5]
    # spans 7, 5, 7, 9, 5, 5 over 1, 2, 3, 1, 2, 1 links: 2 (16 * 128) (16 S)^2 per link
    expect = 2 * 2048 * 256 * (49 * 1 + 25 * 2 + 49 * 3 + 81 * 1 + 25 * 2 + 25 * 1)
    assert bench.tsqr_algorithmic_flops(model, 16) == expect
    assert abs(expect - 0.4215e9) < 1e6
    # and their bytes: every (16 * 128) x (16 S) unfolding read once in float32
    assert bench.tsqr_algorithmic_bytes(model, 16) == 4 * 2048 * 16 * (7 + 5 * 2 + 7 * 3 + 9 + 5 * 2 + 5)


def test_tt_dense_rel_err_matches_densified():
    n = [6, 7, 5, 4]
    a = synth.random_index_bumps_tt(n, 3, seed=11)
    b = synth.random_index_bumps_tt(n, 2, seed=12)
    P = tt.densify(b)
    ref = float(np.linalg.norm(tt.densify(a) - P) / np.linalg.norm(P))
    assert abs(bench.tt_dense_rel_err(a, P) - ref) < 1e-9
    assert bench.tt_dense_rel_err(b, P) < 1e-7
    assert math.isfinite(bench.tt_dense_rel_err([c.astype(np.float32) for c in a], P))


def test_fullgrid_bytes_count_the_fused_passes():
    """Config 2's F = 0.95 I + 0.05 U has no L shears: the full-grid filter
    makes one fused pass per axis and one likelihood-moments pass, each a read
    and a write of the 2^28-cell float32 density."""
    m = synth.config2()
    assert bench.fullgrid_bytes_per_step(m) == 2 ** 28 * 4 * 2 * (4 + 1)
    # a lower-triangular coupling forces the per-operation sequence
    m2 = synth.config2()
    m2.F = np.array(m2.F)
    m2.F[3, 0] = 0.02
    n_ops = len(bench.ldu_ops(m2.F))
    assert bench.fullgrid_bytes_per_step(m2) > 2 ** 28 * 4 * 2 * (4 + 1)
    assert n_ops > 6


def test_tt_pairs_rel_err_matches_densified():
    import bench
    rng = np.random.default_rng([51])
    cores = [rng.standard_normal(s) for s in [(1, 5, 3), (3, 4, 1), (1, 6, 2), (2, 3, 1)]]
    pairs = [rng.standard_normal((5, 4)), rng.standard_normal((6, 3))]
    from oracle import tt
    T = tt.densify(cores)
    P = np.einsum("ab,cd->abcd", pairs[0], pairs[1])
    ref = np.linalg.norm(T - P) / np.linalg.norm(P)
    assert abs(bench.tt_pairs_rel_err(cores, pairs) - ref) < 1e-10
