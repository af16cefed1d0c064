"""The operator entry point that allocates no GPU memory, checked against the
handle-based one.

It lives in its own file, collected last, so a stopped-at-first-failure run
has run every other test before it; it also passes alone in a fresh process
(the first call on a device looks up its scratch array's address)."""
import numpy as np
import pytest

import stokes_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ragged():
    pores = [si.circle_curve((-1.5, 0.1), 0.15, 17), si.circle_curve((0.0, -0.3), 0.2, 50),
             si.circle_curve((1.4, 0.25), 0.12, 33)]
    return si.assemble_geometry(pores, si.superellipse_curve(3.0, 1.0, 203), (3.0, 1.0, 8))


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float64, device="cuda:0")


@pytest.mark.parametrize("which", ["pipe10", "ragged"])
def test_noalloc_matvec_matches_the_handle_matvec_on_two_calls(which):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1609_04484_gb300 as S
    g = si.cached_geometry("pipe10", 0) if which == "pipe10" else _ragged()
    arrs = [_dev(a) for a in (g.nodes, g.normals, g.weights, g.curvature)]
    centres = np.ascontiguousarray(g.centres).reshape(-1)
    stream = torch.cuda.current_stream().cuda_stream
    with S.Geometry(g, stream=stream) as G:
        for seed in (1, 2):          # two calls in a row: nothing stale carries over
            sig = _dev(si.random_density(g, seed))
            y_ref = torch.empty_like(sig)
            S.stokes_matvec(G.handle, sig, y_ref, S.STOKES_FP64)
            y = torch.full_like(sig, float("nan"))
            code = S.stokes_matvec_noalloc(*arrs, g.offsets, g.n_comp, g.outer_comp, centres, sig, y, stream)
            assert code == S.STOKES_OK
            torch.cuda.synchronize()
            err = (torch.linalg.norm(y - y_ref) / torch.linalg.norm(y_ref)).item()
            assert err < 1e-12


def test_noalloc_rejects_host_arrays_and_oversize_problems():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1609_04484_gb300 as S
    g = si.cached_geometry("pipe10", 0)
    centres = np.ascontiguousarray(g.centres).reshape(-1)
    host = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
            for a in (g.nodes, g.normals, g.weights, g.curvature)]
    sig = si.random_density(g, 1).reshape(-1)
    y = np.empty_like(sig)
    assert S.stokes_matvec_noalloc(*host, g.offsets, g.n_comp, g.outer_comp, centres, sig, y) == S.STOKES_EINVAL
    # 2.5 million nodes need more than the 32 MiB scratch array even unsplit
    n = 2_500_000
    off = np.array([0, n], dtype=np.int64)
    z2 = torch.zeros(2 * n, dtype=torch.float64, device="cuda:0")
    z1 = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    code = S.stokes_matvec_noalloc(z2, z2, z1, z1, off, 1, 0, np.zeros(2), z2, torch.empty_like(z2))
    assert code == S.STOKES_EINVAL
