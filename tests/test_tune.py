"""Launch-shape autotuner of the pair kernels.

CPU: the process-wide cache (insert, lookup by size class, JSON-lines file
round trip, rejection of malformed or stale lines) through the C ABI.
GPU: every compiled shape of every pair kernel computes the same operator
(against the CPU oracle), and the tuner picks a shape that is then used.
"""
import json

import numpy as np
import pytest




@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    b = __graft_entry__._build_module()
    if not b.LIB.exists():
        b.build()
    import paper_1609_04484_gb300 as S
    S.stokes_tune_cache_clear()
    yield S
    S.stokes_tune_cache_clear()


def test_variants_are_listed(S):
    for prec in (S.STOKES_FP64, S.STOKES_FP32, S.STOKES_DF64):
        n = S.stokes_pair_shape_count(prec)
        assert n >= 3
        shapes = [S.stokes_pair_shape_info(prec, v) for v in range(n)]
        assert len(set(shapes)) == n
        for th, tpt, tile in shapes:
            assert th % 32 == 0 and tpt >= 1 and tile >= th
    with pytest.raises(S.StokesError):
        S.stokes_pair_shape_info(S.STOKES_FP32, 99)
    assert S.lib.stokes_pair_shape_count(7) == S.STOKES_EINVAL


def test_cache_size_classes_and_file_round_trip(S, tmp_path):
    S.stokes_tune_cache_clear()
    assert S.stokes_tune_cache_lookup(S.STOKES_FP32, 1000, 1000)[0] == -1
    S.stokes_tune_cache_insert(S.STOKES_FP32, 136192, 136192, 1, 8, 14.5)
    S.stokes_tune_cache_insert(S.STOKES_DF64, 1152, 4096, 2, 2, 0.25)
    # same size class: ceil(log2 N) = 18 for 131073..262144
    assert S.stokes_tune_cache_lookup(S.STOKES_FP32, 131073, 262144) == (1, 8, 14.5)
    assert S.stokes_tune_cache_lookup(S.STOKES_FP32, 131072, 136192)[0] == -1
    assert S.stokes_tune_cache_lookup(S.STOKES_DF64, 2048, 4096)[:2] == (2, 2)
    path = tmp_path / "tune.jsonl"
    S.stokes_tune_cache_save(path)
    lines = [json.loads(l) for l in path.read_text().splitlines()]
    assert len(lines) == 2
    for l in lines:
        assert (l["threads"], l["targets_per_thread"], l["tile"]) == \
            S.stokes_pair_shape_info(l["precision"], l["variant"])
    S.stokes_tune_cache_clear()
    assert S.stokes_tune_cache_lookup(S.STOKES_FP32, 136192, 136192)[0] == -1
    assert S.stokes_tune_cache_load(path) == 2
    assert S.stokes_tune_cache_lookup(S.STOKES_FP32, 136192, 136192) == (1, 8, 14.5)
    S.stokes_tune_cache_clear()


def test_cache_load_skips_bad_lines(S, tmp_path):
    S.stokes_tune_cache_clear()
    th, tpt, tile = S.stokes_pair_shape_info(S.STOKES_FP32, 1)
    good = {"precision": 1, "log2_sources": 11, "log2_targets": 11, "variant": 1, "threads": th,
            "targets_per_thread": tpt, "tile": tile, "ctas_per_sm": 4, "ms": 0.1}
    stale = dict(good, log2_sources=12, tile=tile + 1)        # shape of another build
    unknown = dict(good, log2_sources=13, variant=99)
    badprec = dict(good, log2_sources=14, precision=5)
    badcps = dict(good, log2_sources=15, ctas_per_sm=0)
    text = "\n".join([json.dumps(good), "not json", json.dumps(stale), json.dumps(unknown),
                      json.dumps(badprec), json.dumps(badcps), '{"precision": 1}', ""])
    path = tmp_path / "mixed.jsonl"
    path.write_text(text)
    assert S.stokes_tune_cache_load(path) == 1
    assert S.stokes_tune_cache_lookup(1, 2048, 2048)[:2] == (1, 4)
    for ln in (12, 13, 15):
        assert S.stokes_tune_cache_lookup(1, 2 ** ln, 2048)[0] == -1
    with pytest.raises(S.StokesError):
        S.stokes_tune_cache_load(tmp_path / "missing.jsonl")
    with pytest.raises(S.StokesError):
        S.stokes_tune_cache_insert(S.STOKES_FP32, 10, 10, 99, 4)
    with pytest.raises(S.StokesError):
        S.stokes_tune_cache_insert(S.STOKES_FP32, 0, 10, 0, 4)
    S.stokes_tune_cache_clear()


def test_shape_calls_reject_null_handle(S):
    assert S.lib.stokes_set_pair_shape(None, S.STOKES_FP32, 0, 4) == S.STOKES_EINVAL
    assert S.lib.stokes_autotune(None, S.STOKES_FP32, 1, None, None, None) == S.STOKES_EINVAL


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------

def _gpu_S(S):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _rel(a, b):
    a, b = np.asarray(a).reshape(-1), np.asarray(b).reshape(-1)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.gpu
@pytest.mark.parametrize("prec,bound", [("FP64", 1e-12), ("DF64", 1e-12), ("FP32", 2e-6)])
def test_every_shape_matches_oracle(S, prec, bound):
    """A ragged geometry (component sizes 17, 50, 33, 203: tails in every
    tile) through every (variant, ctas_per_sm) of the pair kernel."""
    _gpu_S(S)
    import oracle as O
    import stokes_inputs as si
    pores = [si.circle_curve((-1.5, 0.1), 0.15, 17), si.circle_curve((0.0, -0.3), 0.2, 50),
             si.circle_curve((1.4, 0.25), 0.12, 33)]
    g = si.assemble_geometry(pores, si.superellipse_curve(3.0, 1.0, 203), (3.0, 1.0, 8))
    sig = si.random_density(g, 4).reshape(-1)
    ref = O.matvec(g, sig)
    T = si.interior_targets(g, 300, min_dist=0.05, seed=2)
    uref = O.velocity(g, sig, T)
    p = getattr(S, "STOKES_" + prec)
    with S.Geometry(g) as G:
        for v in range(S.stokes_pair_shape_count(p)):
            for cps in (1, 2, 8):
                S.stokes_set_pair_shape(G.handle, p, v, cps)
                assert S.stokes_get_pair_shape(G.handle, p, g.n_nodes) == (v, cps)
                y = np.empty_like(sig)
                S.stokes_matvec(G.handle, sig, y, p)
                assert _rel(y, ref) < bound, (v, cps)
                u = np.empty(T.size)
                S.stokes_eval_velocity(G.handle, sig, T.reshape(-1), u, p)
                assert _rel(u, uref) < bound, (v, cps)


@pytest.mark.gpu
def test_autotune_picks_a_shape_and_caches_it(S, tmp_path):
    _gpu_S(S)
    import stokes_inputs as si
    g = si.cached_geometry("pipe10", 0)
    S.stokes_tune_cache_clear()
    sig = si.random_density(g, 1).reshape(-1)
    with S.Geometry(g) as G:
        y0 = np.empty_like(sig)
        S.stokes_matvec(G.handle, sig, y0, S.STOKES_DF64)
        v, cps, ms = S.stokes_autotune(G.handle, S.STOKES_DF64, reps=2)
        assert 0 <= v < S.stokes_pair_shape_count(S.STOKES_DF64) and cps in (2, 4, 8) and ms > 0
        assert S.stokes_get_pair_shape(G.handle, S.STOKES_DF64, g.n_nodes) == (v, cps)
        y1 = np.empty_like(sig)
        S.stokes_matvec(G.handle, sig, y1, S.STOKES_DF64)
        assert _rel(y1, y0) < 1e-13
    # a new handle of the same size class takes the cached shape
    with S.Geometry(g) as G2:
        assert S.stokes_get_pair_shape(G2.handle, S.STOKES_DF64, g.n_nodes) == (v, cps)
        S.stokes_set_pair_shape(G2.handle, S.STOKES_DF64, 0, 4)
        assert S.stokes_get_pair_shape(G2.handle, S.STOKES_DF64, g.n_nodes) == (0, 4)
        S.stokes_set_pair_shape(G2.handle, S.STOKES_DF64, -1)
        assert S.stokes_get_pair_shape(G2.handle, S.STOKES_DF64, g.n_nodes) == (v, cps)
    path = tmp_path / "t.jsonl"
    S.stokes_tune_cache_save(path)
    S.stokes_tune_cache_clear()
    assert S.stokes_tune_cache_load(path) == 1
    assert S.stokes_tune_cache_lookup(S.STOKES_DF64, g.n_nodes, g.n_nodes)[:2] == (v, cps)
    S.stokes_tune_cache_clear()
