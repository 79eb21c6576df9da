"""CPU-side tests of libpcx: the C ABI loads and exports every declared
symbol, and the host-only entry points (sampling, Rayleigh-Ritz solver)
agree with the oracle.  No kernel is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest
import scipy.linalg

import workloads as wl
from oracle import permittivity

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pcx():
    from paper_2511_17107_gb300 import build, pcx as binding
    build.build()
    binding.lib()
    return binding


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "pcx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(pcx_\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_symbol(pcx):
    names = _declared_functions()
    assert "pcx_apply" in names and "pcx_solve" in names and len(names) >= 15
    lib = pcx.lib()
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(pcx.exported_symbols())


@pytest.mark.parametrize("m,seed", [(6, 0), (24, 1), (48, 2)])
def test_rr_eig_matches_lapack(pcx, m, seed):
    """Generalised Hermitian eigenproblem of the Rayleigh-Ritz step vs
    scipy.linalg.eigh (LAPACK)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    ga = a @ a.conj().T + np.diag(np.linspace(0.1, 50, m))
    b = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    gb = b @ b.conj().T / m + np.eye(m)
    th, c = pcx.pcx_rr_eig(ga, gb, 1e-14)
    want = scipy.linalg.eigh(ga, gb, eigvals_only=True)
    assert c.shape == (m, m)
    np.testing.assert_allclose(th, want, rtol=1e-11)
    np.testing.assert_allclose(c.conj().T @ gb @ c, np.eye(m), atol=1e-10)
    np.testing.assert_allclose(c.conj().T @ ga @ c, np.diag(th), atol=1e-9 * th.max())


def test_rr_eig_drops_dependent_directions(pcx):
    """A metric of rank 4 in 6 dimensions leaves a 4-dimensional problem."""
    rng = np.random.default_rng(3)
    v = rng.standard_normal((6, 4)) + 1j * rng.standard_normal((6, 4))
    gb = v @ v.conj().T
    ga = v @ np.diag([1.0, 2.0, 3.0, 4.0]) @ v.conj().T
    th, c = pcx.pcx_rr_eig(ga, gb, 1e-10)
    assert c.shape == (6, 4)
    np.testing.assert_allclose(c.conj().T @ gb @ c, np.eye(4), atol=1e-9)


STRUCTS = [
    ("sc", wl.sc_gyro_sphere),
    ("fcc", wl.fcc_air_spheres),
    ("diamond", wl.diamond_rods),
    ("woodpile", wl.woodpile),
    ("random", lambda: wl.random_inclusions(7)),
    ("gyroid", lambda: wl.Structure("g", wl.BCC.copy(), np.stack([wl.VACUUM, wl.paper_anisotropic(16.0)]), 0,
                                    [wl.Shape(wl.SHAPE_GYROID, 1, (1.1, 0))])),
]


@pytest.mark.parametrize("name,maker", STRUCTS)
@pytest.mark.parametrize("n", [8, 16])
def test_sampling_matches_oracle(pcx, name, maker, n):
    """Row a1: material index of every staggered sample point (bit-exact)
    and the packed cell blocks (FP64 inverse permittivities)."""
    s = maker()
    blocks, ids, bad = pcx.pcx_sample_host(s, n)
    for i, w in enumerate(permittivity.POINT_SETS):
        want = permittivity.material_ids(s, n, w).ravel()
        assert np.array_equal(ids[i], want), (name, w, int(np.sum(ids[i] != want)))
    ob = permittivity.cell_blocks(s, n).reshape(-1, 3, 3)
    packed = np.stack([ob[:, 0, 0].real, ob[:, 1, 1].real, ob[:, 2, 2].real, ob[:, 0, 1].real, ob[:, 0, 1].imag,
                       ob[:, 0, 2].real, ob[:, 0, 2].imag, ob[:, 1, 2].real, ob[:, 1, 2].imag], axis=1)
    np.testing.assert_allclose(blocks, packed, rtol=1e-14, atol=1e-16)
    hpd = permittivity.cell_min_eigenvalue(ob.reshape(n, n, n, 3, 3)).ravel() > 0
    assert bad == (-1 if hpd.all() else int(np.argmin(hpd)))


def test_non_hpd_cell_reported(pcx):
    strong = np.linalg.inv(np.array([[1.0, 0.95j, 0], [-0.95j, 1.0, 0], [0, 0, 1.0]]))
    weak = np.diag([40.0, 40.0, 40.0]).astype(complex)
    s = wl.Structure("t", wl.SC.copy(), np.stack([weak, strong]), 0,
                     [wl.Shape(wl.SHAPE_BOX, 1, (0.3, 0.3, 0.3, 0.7, 0.7, 0.7))])
    _, _, bad = pcx.pcx_sample_host(s, 8)
    ob = permittivity.cell_blocks(s, 8)
    hpd = permittivity.cell_min_eigenvalue(ob).ravel() > 0
    assert bad == int(np.argmin(hpd)) and bad >= 0


@pytest.mark.parametrize("n,m,lat", [(12, 1, wl.SC), (6, 1, wl.SC), (8, 6, wl.SC), (8, 5, wl.SC),
                                     (8, 1, np.zeros((3, 3)))])
def test_invalid_setup_rejected(pcx, n, m, lat):
    s = wl.sc_gyro_sphere()
    s.lattice = lat
    with pytest.raises(pcx.PcxError) as ei:
        pcx.pcx_sample_host(s, n, stencil_m=m)
    assert ei.value.status == pcx.PCX_EINVAL


def test_cnn_parameter_count_matches_oracle_layout():
    import re
    from oracle import learned
    from paper_2511_17107_gb300 import pcx as binding
    assert binding.PCX_CNN_NPARAMS == learned.param_count(binding.PCX_CNN_HIDDEN)
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "pcx.h")).read()
    assert re.search(r"#define PCX_CNN_HIDDEN 8\b", hdr)


def test_gram_path_setting_is_validated(pcx):
    """pcx_set_gram_path takes the three documented values and rejects
    others without changing the current choice (host-side state only)."""
    assert pcx.pcx_get_gram_path() == pcx.PCX_GRAM_AUTO
    for path in (pcx.PCX_GRAM_TENSOR, pcx.PCX_GRAM_FP32, pcx.PCX_GRAM_AUTO):
        pcx.pcx_set_gram_path(path)
        assert pcx.pcx_get_gram_path() == path
    for bad in (-1, 3, 7):
        with pytest.raises(pcx.PcxError):
            pcx.pcx_set_gram_path(bad)
    assert pcx.pcx_get_gram_path() == pcx.PCX_GRAM_AUTO



def test_crossdof_setup_validation(pcx):
    """m_kind takes PCX_M_TRIVIAL or PCX_M_CROSSDOF; M_CrossDoF needs the
    material ids of a structure, so caller-supplied cell blocks are refused
    (host-side validation, before any device work)."""
    s = wl.sc_gyro_sphere()
    blocks, ids, bad = pcx.pcx_sample_host(s, 8, m_kind=pcx.PCX_M_CROSSDOF)
    assert bad == -1 and blocks.shape == (8 ** 3, 9)
    with pytest.raises(pcx.PcxError) as ei:
        pcx.pcx_sample_host(s, 8, m_kind=7)
    assert ei.value.status == pcx.PCX_EINVAL
    with pytest.raises(pcx.PcxError) as ei:
        pcx.pcx_sample_host(s, 8, m_kind=pcx.PCX_M_CROSSDOF, cell_blocks=blocks)
    assert ei.value.status == pcx.PCX_EINVAL


def test_crossdof_sec33_conditions(pcx):
    """M_CrossDoF's HPD check follows Sec. 3.3: Assumption 3.1 (eps_1 in
    (0, 1]) with a zero off-diagonal shared by every material (3.3) or a
    strictly diagonally dominant assembled matrix (3.2).  Where the check
    passes, the oracle's dense M_CrossDoF is HPD; a material outside (0, 1]
    and a dense rotated tensor that is not diagonally dominant are reported
    as unproven."""
    from oracle import crossdof
    n = 8
    # the paper's anisotropic eps_1 (zero xz and yz entries, SDD) on a BCC gyroid
    paper = wl.Structure("g", wl.BCC.copy(), np.stack([wl.VACUUM, wl.paper_anisotropic(16.0)]), 0,
                         [wl.Shape(wl.SHAPE_GYROID, 1, (1.1, 0))])
    assert pcx.pcx_sample_host(paper, n, m_kind=pcx.PCX_M_CROSSDOF)[2] == -1
    m = crossdof.CrossDofM(paper, 6).dense()
    assert np.linalg.eigvalsh(0.5 * (m + m.conj().T)).min() > 0
    # a dense, weakly diagonal eps_1 (every off-diagonal nonzero, SDD fails) ...
    rng = np.random.default_rng(2)
    u = wl.seeded_unitary(rng)
    inv = (u * np.array([0.06, 0.5, 0.95])) @ u.conj().T
    dense = wl.Structure("d", wl.SC.copy(), np.stack([wl.VACUUM, np.linalg.inv(inv)]), 0,
                         [wl.Shape(wl.SHAPE_SPHERE, 1, (0.5, 0.5, 0.5, 0.3))])
    assert np.all(np.abs(inv[np.triu_indices(3, 1)]) > 1e-3)
    assert pcx.pcx_sample_host(dense, n, m_kind=pcx.PCX_M_CROSSDOF)[2] >= 0
    # ... and a material whose eps_1 has an eigenvalue above 1 (eps below vacuum)
    weak = wl.Structure("w", wl.SC.copy(), np.stack([wl.VACUUM, 0.5 * wl.VACUUM]), 0,
                        [wl.Shape(wl.SHAPE_SPHERE, 1, (0.5, 0.5, 0.5, 0.3))])
    assert pcx.pcx_sample_host(weak, n, m_kind=pcx.PCX_M_CROSSDOF)[2] == 0
    # the same structures under M_Trivial are judged cell by cell instead
    assert pcx.pcx_sample_host(dense, n)[2] == -1


def test_host_entries_reject_bad_arguments_before_any_device_work(pcx):
    """The host-buffer entries check their arguments on the host: a NULL
    context, negative counts or strides, and NULL or misaligned buffers give
    PCX_EINVAL without touching a device (so this runs without a GPU)."""
    lib = pcx.lib()
    k = np.zeros(3)
    kp = k.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    buf = np.zeros(64, dtype=np.complex64)
    p = ctypes.c_void_p(buf.ctypes.data)
    assert lib.pcx_apply_kbatch_host(None, kp, 1, 0.0, p, 0, p, 0, 1, 1, None) == pcx.PCX_EINVAL
    assert lib.pcx_apply_host(None, kp, 0.0, p, p, 1, 1, None) == pcx.PCX_EINVAL
    assert lib.pcx_apply_kbatch(None, kp, 1, 0.0, p, p, 1, 1, None) == pcx.PCX_EINVAL
