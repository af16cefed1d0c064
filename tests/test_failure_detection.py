"""Failure detection of the persistent kernels' grid barriers, without a GPU
fault: the barrier's poll limit is taken from STOKES_WAIT_POLLS at each
launch, so a limit of zero makes every early-arriving CTA give up at once.
The kernel then raises its sticky error flag and every CTA returns at its
next barrier; the host turns the flag into STOKES_ECUDA with a message, and
a fresh handle works normally afterwards."""
import os

import numpy as np
import pytest

import oracle as O
import stokes_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture
def S():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1609_04484_gb300 as S
    return S


@pytest.fixture
def no_patience(monkeypatch):
    """Run the body with the barrier poll limit at zero; restore after."""
    def on():
        monkeypatch.setenv("STOKES_WAIT_POLLS", "0")

    def off():
        monkeypatch.delenv("STOKES_WAIT_POLLS", raising=False)
    yield on, off
    os.environ.pop("STOKES_WAIT_POLLS", None)


def _two_grid_lu_handle(S, g):
    G = S.Geometry(g)
    S.stokes_precond_setup_twogrid_ex(G.handle, 2, S.STOKES_TG_COARSE_LU)
    return G


def test_triangular_solve_barrier_timeout_is_reported(S, no_patience):
    on, off = no_patience
    g = si.pipe10_geometry(0, n_outer=256, n_pores=4, n_per_pore=32)
    r = torch.tensor(si.random_density(g, 5).reshape(-1), device="cuda:0")
    z = torch.empty_like(r)
    G = _two_grid_lu_handle(S, g)
    try:
        on()
        with pytest.raises(S.StokesError) as e:
            S.stokes_precond_apply(G.handle, r, z)
        assert e.value.code == S.STOKES_ECUDA and "timed out" in str(e.value)
    finally:
        off()
        G.close()
    # a fresh handle is unaffected and matches the oracle's two-grid apply
    # (float coarse factors: 1e-3, as in the two-grid parity tests)
    G = _two_grid_lu_handle(S, g)
    try:
        S.stokes_precond_apply(G.handle, r, z)
        torch.cuda.synchronize()
        ref = O.TwoGrid(g, 2).apply(r.cpu().numpy())
        assert np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-3
    finally:
        G.close()


def test_panel_factorisation_barrier_timeout_is_reported(S, no_patience, monkeypatch):
    on, off = no_patience
    monkeypatch.setenv("STOKES_TG_PANEL", "coop")
    g = si.pipe10_geometry(0, n_outer=256, n_pores=4, n_per_pore=32)
    G = S.Geometry(g)
    try:
        on()
        with pytest.raises(S.StokesError) as e:
            S.stokes_precond_setup_twogrid_ex(G.handle, 2, S.STOKES_TG_COARSE_LU)
        assert e.value.code == S.STOKES_ECUDA and "timed out" in str(e.value)
        off()
        # the same handle sets up again (each setup starts a fresh barrier)
        S.stokes_precond_setup_twogrid_ex(G.handle, 2, S.STOKES_TG_COARSE_INVERSE)
    finally:
        off()
        G.close()
