"""The per-iteration residual history of pcx_solve (opts.res_history) and the
M_CrossDoF setup without the Sec. 3.3 proof (crossdof_unchecked), through
the C ABI."""
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


@pytest.mark.parametrize("prec", [0, 1])
def test_residual_history_records_every_iteration(pcx, prec):
    """One entry per LOBPCG iteration, each the worst wanted residual of that
    iteration: the count matches the iteration counters, the last entry is the
    converged one and the history falls overall."""
    n, nev = 16, 6
    s = wl.sc_gyro_sphere()
    k = wl.config_k(s.name)[0]
    ctx = pcx.setup_structure(s, n)
    hist = np.full(4000, np.nan)
    stats = pcx.pcx_solve_stats()
    ev, res, its, st = pcx.pcx_solve(ctx, [k], nev, 1e-8, block=nev + 4, precision=prec, stats=stats,
                                     res_history=hist, penalty_tol=-1.0)
    assert st == pcx.PCX_OK
    m = stats.history_len
    assert m >= stats.iters_fp32 + stats.iters_fp64 >= 1
    h = hist[:m]
    assert np.all(np.isfinite(h)) and np.all(np.isnan(hist[m:]))
    assert h[-1] <= 1e-8 and h[-1] == pytest.approx(np.max(res), rel=1e-12)
    assert h[0] > 1e3 * h[-1]
    # a cap shorter than the run: entries stop at the cap, the count is the cap
    short = np.full(5, np.nan)
    pcx.pcx_solve(ctx, [k], nev, 1e-8, block=nev + 4, precision=prec, stats=stats, res_history=short,
                  penalty_tol=-1.0)
    assert stats.history_len == 5 and np.all(np.isfinite(short))


def test_crossdof_unchecked_accepts_what_the_proof_refuses(pcx):
    """The Sec. 4.4 material (inverse permittivity with eigenvalues 1e-1,
    1e-3, 1e-5 and no zero off-diagonal) fails the sufficient conditions of
    Sec. 3.3: M_CrossDoF is refused with PCX_ENOTHPD unless the unchecked
    build is asked for; M_Trivial is accepted either way."""
    s = wl.ill_conditioned_sphere()
    with pytest.raises(pcx.PcxError) as e:
        pcx.setup_structure(s, 32, m_kind=pcx.PCX_M_CROSSDOF)
    assert e.value.status == pcx.PCX_ENOTHPD
    ctx = pcx.setup_structure(s, 32, m_kind=pcx.PCX_M_CROSSDOF, crossdof_unchecked=True)
    x = torch.from_numpy(wl.random_block(1, 32, seed=3)).cuda()
    y = torch.empty_like(x)
    pcx.pcx_apply(ctx, wl.config_k(s.name)[0], x, y)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(y)).all()
    pcx.setup_structure(s, 32)
