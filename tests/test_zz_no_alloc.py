"""The operator entry point that allocates no GPU memory, checked against the
CPU oracle and against the handle-based operator.

Callers that cannot allocate (an allocator owning the whole device, paths
where an allocation's device synchronisation is not allowed) use
stokes_matvec_noalloc, whose scratch is a fixed device array inside the
library. This file is collected last, so a stopped-at-first-failure run has
run every other test before it; it also passes alone in a fresh process
(the first call on a device looks up the scratch array's address)."""
import dataclasses

import numpy as np
import pytest

import oracle
import stokes_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ragged():
    pores = [si.circle_curve((-1.5, 0.1), 0.15, 17), si.circle_curve((0.0, -0.3), 0.2, 50),
             si.circle_curve((1.4, 0.25), 0.12, 33)]
    return si.assemble_geometry(pores, si.superellipse_curve(3.0, 1.0, 203), (3.0, 1.0, 8))


def _wall_first(g):
    """The same boundary with the wall stored as component 0."""
    k0 = g.outer_comp
    order = [k0] + [k for k in range(g.n_comp) if k != k0]
    idx = np.concatenate([np.arange(g.offsets[k], g.offsets[k + 1]) for k in order])
    sizes = np.diff(g.offsets)[order]
    return dataclasses.replace(
        g, nodes=g.nodes[idx].copy(), normals=g.normals[idx].copy(), weights=g.weights[idx].copy(),
        curvature=g.curvature[idx].copy(), offsets=np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64),
        outer_comp=0, centres=g.centres[order].copy(), radii=g.radii[order].copy())


def _wall_only():
    return si.assemble_geometry([], si.superellipse_curve(3.0, 1.0, 301), (3.0, 1.0, 8))


def _geometry(which):
    if which == "pipe10":
        return si.cached_geometry("pipe10", 0)
    if which == "ragged":
        return _ragged()
    if which == "wall_first":
        return _wall_first(_ragged())
    return _wall_only()


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float64, device="cuda:0")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("which", ["pipe10", "ragged", "wall_first", "wall_only"])
def test_noalloc_matvec_matches_oracle_and_handle_matvec_on_two_calls(which):
    """Two calls in a row (nothing stale carries over in the shared scratch
    array) against the oracle's matrix-free operator at 1e-12 (the FP64
    operator's parity bound) and against stokes_matvec at 1e-12; the
    library's launch counter sees the call's three kernels."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1609_04484_gb300 as S
    g = _geometry(which)
    arrs = [_dev(a) for a in (g.nodes, g.normals, g.weights, g.curvature)]
    centres = np.ascontiguousarray(g.centres).reshape(-1)
    stream = torch.cuda.current_stream().cuda_stream
    with S.Geometry(g, stream=stream) as G:
        for seed in (1, 2):
            s_h = si.random_density(g, seed).reshape(-1)
            sig = _dev(s_h)
            y_ref = torch.empty_like(sig)
            S.stokes_matvec(G.handle, sig, y_ref, S.STOKES_FP64)
            y = torch.full_like(sig, float("nan"))
            n0 = S.stokes_kernel_launches()
            code = S.stokes_matvec_noalloc(*arrs, g.offsets, g.n_comp, g.outer_comp, centres, sig, y, stream)
            assert code == S.STOKES_OK
            torch.cuda.synchronize()
            assert S.stokes_kernel_launches() - n0 == 3
            y_h = y.cpu().numpy()
            assert _rel(y_h, oracle.matvec(g, s_h)) < 1e-12
            assert _rel(y_h, y_ref.cpu().numpy()) < 1e-12


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
    n0 = S.stokes_kernel_launches()
    assert S.stokes_matvec_noalloc(*host, g.offsets, g.n_comp, g.outer_comp, centres, sig, y) == S.STOKES_EINVAL
    # 2.5 million nodes need more than the 32 MiB scratch array even unsplit
    n = 2_500_000
    off = np.array([0, n], dtype=np.int64)
    z2 = torch.zeros(2 * n, dtype=torch.float64, device="cuda:0")
    z1 = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    code = S.stokes_matvec_noalloc(z2, z2, z1, z1, off, 1, 0, np.zeros(2), z2, torch.empty_like(z2))
    assert code == S.STOKES_EINVAL
    assert S.stokes_kernel_launches() == n0  # rejected before anything ran


def test_noalloc_rejects_another_devices_arrays():
    if not torch.cuda.is_available() or torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    import paper_1609_04484_gb300 as S
    g = si.cached_geometry("pipe10", 0)
    on1 = lambda a: torch.tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float64, device="cuda:1")
    arrs = [on1(a) for a in (g.nodes, g.normals, g.weights, g.curvature)]
    sig = on1(si.random_density(g, 1))
    with torch.cuda.device(0):
        code = S.stokes_matvec_noalloc(*arrs, g.offsets, g.n_comp, g.outer_comp,
                                       np.ascontiguousarray(g.centres).reshape(-1), sig, torch.empty_like(sig))
    assert code == S.STOKES_EINVAL
