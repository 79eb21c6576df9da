"""Failure handling of pcx_solve, with every failure made on the host (no GPU
fault is ever provoked): NaN in the initial block, a rank-deficient initial
block, and an iteration cap that runs out.  Also the warm start that the
initial-block option exists for."""
import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pcx():
    from paper_2511_17107_gb300 import build, pcx as binding
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return binding


def _x0(n, block, seed):
    return torch.from_numpy(wl.random_block(block, n, seed=seed)).cuda()


@pytest.mark.parametrize("prec", [0, 1])
def test_nan_in_initial_block_is_a_numeric_error(pcx, prec):
    n, nev, block = 16, 4, 8
    s = wl.sc_gyro_sphere()
    k = wl.config_k(s.name)[0]
    ctx = pcx.setup_structure(s, n)
    x0 = _x0(n, block, 3)
    x0[2, 1, 3, 4, 5] = complex(float("nan"), 0.0)
    with pytest.raises(pcx.PcxError) as e:
        pcx.pcx_solve(ctx, [k], nev, 1e-8, block=block, precision=prec, x0=x0)
    assert e.value.status == pcx.PCX_ENUMERIC
    # the context stays usable: the same solve from a clean block converges
    ev, res, its, st = pcx.pcx_solve(ctx, [k], nev, 1e-8, block=block, precision=prec, x0=_x0(n, block, 3))
    assert st == pcx.PCX_OK and np.all(res <= 1e-8)


def test_rank_deficient_initial_block_is_a_numeric_error(pcx):
    n, nev, block = 16, 4, 8
    s = wl.sc_gyro_sphere()
    k = wl.config_k(s.name)[0]
    ctx = pcx.setup_structure(s, n)
    x0 = _x0(n, block, 4)
    x0[5] = x0[1]          # two equal columns: a singular Gram matrix
    with pytest.raises(pcx.PcxError) as e:
        pcx.pcx_solve(ctx, [k], nev, 1e-8, block=block, precision=0, x0=x0)
    assert e.value.status == pcx.PCX_ENUMERIC
    assert "rank" in str(e.value)


@pytest.mark.parametrize("prec", [0, 1])
def test_iteration_cap_returns_noconv_with_partial_outputs(pcx, prec):
    """maxit = 3: PCX_ENOCONV, with the last iterate's Ritz values (finite,
    ascending, above the converged ones) and residuals (above tol)
    written."""
    n, nev = 16, 6
    s = wl.sc_gyro_sphere()
    k = wl.config_k(s.name)[0]
    ctx = pcx.setup_structure(s, n)
    ev, res, its, st = pcx.pcx_solve(ctx, [k], nev, 1e-10, block=10, precision=prec, maxit=3,
                                     raise_on_noconv=False)
    assert st == pcx.PCX_ENOCONV
    assert np.all(np.isfinite(ev)) and np.all(np.diff(ev[0]) >= 0)
    assert np.all(np.isfinite(res)) and res.max() > 1e-10
    assert 1 <= its[0] <= 3 + 1
    ref, rres, rits, rst = pcx.pcx_solve(ctx, [k], nev, 1e-10, block=10, precision=prec)
    assert rst == pcx.PCX_OK
    # Rayleigh-Ritz values bound the eigenvalues from above
    assert np.all(ev[0] >= ref[0] * (1 - 1e-9))


def test_warm_start_from_the_previous_k(pcx):
    """Along a band path the eigenvectors of one k are a good start for the
    next: the same eigenvalues (1e-10) in fewer iterations than a cold start."""
    n, nev, block = 16, 8, 12
    s = wl.fcc_air_spheres()
    path = wl.config_k(s.name)
    ctx = pcx.setup_structure(s, n)
    vec = torch.empty((nev, 3, n, n, n), dtype=torch.complex128, device="cuda")
    ev0, res0, its0, st0 = pcx.pcx_solve(ctx, [path[12]], nev, 1e-10, block=block, vec_out=vec)
    assert st0 == pcx.PCX_OK
    cold, _, its_cold, st1 = pcx.pcx_solve(ctx, [path[13]], nev, 1e-10, block=block)
    x0 = torch.cat([vec, _x0(n, block - nev, 9)])
    warm, _, its_warm, st2 = pcx.pcx_solve(ctx, [path[13]], nev, 1e-10, block=block, x0=x0)
    assert st1 == pcx.PCX_OK and st2 == pcx.PCX_OK
    np.testing.assert_allclose(warm[0], cold[0], rtol=1e-10)
    assert its_warm[0] < its_cold[0], (its_warm, its_cold)
