"""Host-only checks of the C ABI (no GPU needed): the library builds for sm_103a,
loads, exports every entry point ``include/qtm.h`` declares, and rejects invalid
problem statements before touching the GPU."""

import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1810_03047_gb300 import qtm as Q
from paper_1810_03047_gb300 import systems as S

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "qtm.h")


def declared_entry_points():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(qtm_[a-z_]+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_header_declares_the_binding_exports():
    assert set(declared_entry_points()) == set(Q.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = Q.lib()
    for name in declared_entry_points():
        assert hasattr(L, name), name


def test_version_and_status_strings():
    assert "sm_103a" in Q.qtm_version()
    assert Q.qtm_status_string(Q.QTM_ERR_ARG) == "QTM_ERR_ARG"
    assert Q.qtm_status_string(Q.QTM_ERR_UNSUPPORTED) == "QTM_ERR_UNSUPPORTED"


def _expect_error(prob, status, fragment, **kw):
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_create(prob, **kw)
    assert ei.value.status == status
    assert fragment in str(ei.value)


def test_rejects_non_hermitian_h():
    prob = S.two_level_driven()
    H = prob.H.toarray()
    H[0, 1] += 0.1
    _expect_error(prob.with_(H=sp.csr_matrix(H)), Q.QTM_ERR_ARG, "Hermitian")


def test_rejects_non_hermitian_observable():
    prob = S.two_level_driven()
    _expect_error(prob.with_(A=[S.sigma_minus()]), Q.QTM_ERR_ARG, "A[0] is not Hermitian")


def test_rejects_bad_time_grid():
    prob = S.two_level_driven()
    _expect_error(prob.with_(t=np.array([0.0, 1.0, 1.0])), Q.QTM_ERR_ARG, "strictly increasing")
    _expect_error(prob.with_(t=np.array([0.0, np.nan])), Q.QTM_ERR_ARG, "non-finite")


def test_rejects_bad_tolerances_and_limits():
    prob = S.two_level_driven()
    _expect_error(prob.with_(rtol=0.0), Q.QTM_ERR_ARG, "rtol")
    _expect_error(prob.with_(atol=-1.0), Q.QTM_ERR_ARG, "rtol")
    _expect_error(prob.with_(max_steps=0), Q.QTM_ERR_ARG, "max_steps")


def test_rejects_bad_csr():
    prob = S.two_level_driven()
    bad = sp.csr_matrix(prob.C[0])
    bad.indices = bad.indices.copy()
    bad.indices[0] = 7
    _expect_error(prob.with_(C=[bad]), Q.QTM_ERR_ARG, "out of range")
    _expect_error(prob.with_(C=[S.destroy(3)]), Q.QTM_ERR_ARG, "differs from dim")


def test_rejects_bad_state():
    prob = S.two_level_driven()
    _expect_error(prob.with_(psi0=np.zeros(2, complex)), Q.QTM_ERR_ARG, "psi0 is zero")
    _expect_error(prob.with_(psi0=np.array([np.inf, 0], complex)), Q.QTM_ERR_ARG, "non-finite psi0")


def test_rejects_unknown_precision_and_flags():
    prob = S.two_level_driven()
    _expect_error(prob, Q.QTM_ERR_ARG, "precision", precision=99)


def test_too_large_dimension_is_unsupported():
    prob = S.ising_chain(11)  # N = 2048: ten state vectors no longer fit in shared memory
    _expect_error(prob, Q.QTM_ERR_UNSUPPORTED, "dimension")


def test_last_error_without_context():
    with pytest.raises(Q.QtmError):
        Q.qtm_create(S.two_level_driven().with_(rtol=-1.0))
    assert "rtol" in Q.qtm_last_error(None)


@pytest.mark.parametrize("name,dts", [
    ("paper_unitary", [0.0, 0.1, 1.0, 10.0]),
    ("jaynes_cummings_driven", [0.1, 2.5]),
    ("purcell_qubit", [0.1, 1.0, 20.0]),          # nu dt up to ~1e4: 18 squarings
    ("dense_random", [0.1]),
])
def test_host_propagator_matches_scipy_expm(name, dts):
    """The exponential method's ladder arithmetic (scaling and squaring of a degree-12
    Taylor polynomial, on the host) against scipy's Pade-based expm of the same M
    (formed here from H and the C_n)."""
    import scipy.linalg
    prob = S.by_name(name, N=64) if name == "dense_random" else S.by_name(name)
    H = prob.H.toarray()
    M = -1j * H
    for c in prob.C:
        c = c.toarray()
        M = M - 0.5 * c.conj().T @ c
    for dt in dts:
        got = Q.qtm_propagator(prob, dt)
        ref = scipy.linalg.expm(M * dt)
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(got - ref).max() <= 1e-12 * scale, (name, dt, np.abs(got - ref).max())


def test_host_propagator_semigroup_and_errors():
    prob = S.purcell_qubit()
    a, b = Q.qtm_propagator(prob, 0.3), Q.qtm_propagator(prob, 0.45)
    np.testing.assert_allclose(a @ b, Q.qtm_propagator(prob, 0.75), atol=1e-13)
    for dt in (-1.0, np.nan, np.inf):
        with pytest.raises(Q.QtmError) as ei:
            Q.qtm_propagator(prob, dt)
        assert ei.value.status == Q.QTM_ERR_ARG
