"""Time-dependent Hamiltonians on the GPU (run with ``-m gpu``):
H(t) = H + sum_k a_k cos(omega_k t + phi_k) H_k (Sec. 3: mpi_main takes an extra
function for a time-dependent Hamiltonian), set with qtm_set_drive.

complex128 and double-float are held to the trajectory-by-trajectory bars of the
static parity tests against the FP64 oracle (which evaluates the same terms at
every stage time); complex64 statistically; the dephasing qubit additionally
against its closed form on the GPU's own jump times."""

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1810_03047_gb300 import qtm as Q
from paper_1810_03047_gb300 import systems as S

from test_gpu_parity import PRECS, _within_statistics, compare, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec_name,prec", PRECS)
@pytest.mark.parametrize("name,n", [("driven_dephasing_qubit", 300), ("jaynes_cummings_pulsed", 403)])
def test_driven_parity_with_oracle(orc, prec_name, prec, name, n):
    prob = S.by_name(name, ntraj=n)
    g = gpu_run(prob, n, precision=prec)
    o = oracle_run(orc, prob, n)
    compare(g, o, n, precision=prec)


def test_dephasing_closed_form_on_gpu_jumps():
    """<sigma_x> = (-1)^N cos 2F and <sigma_y> = (-1)^N sin 2F per trajectory, with
    N counted from the GPU's own jump times (rtol 1e-8: within 1e-6)."""
    prob = S.driven_dephasing_qubit(ntraj=500)
    g = gpu_run(prob, 500, precision=Q.QTM_PREC_DF64)
    (_, a, w, ph), = prob.drive
    F = (a / w) * (np.sin(w * prob.t + ph) - np.sin(ph))
    assert g["n_jumps"].sum() > 250
    for i in range(500):
        jt = g["jump_t"][i, :g["n_jumps"][i]]
        N = (jt[None, :] <= prob.t[:, None]).sum(axis=1)
        np.testing.assert_allclose(g["obs"][i, :, 0], (-1.0) ** N * np.cos(2 * F), atol=1e-6)
        np.testing.assert_allclose(g["obs"][i, :, 1], (-1.0) ** N * np.sin(2 * F), atol=1e-6)


def test_driven_complex64_statistics(orc):
    prob = S.jaynes_cummings_pulsed(ntraj=403)
    g = gpu_run(prob, 403, precision=Q.QTM_PREC_C64)
    o = oracle_run(orc, prob, 403)
    assert np.mean(g["n_jumps"] == o["n_jumps"]) >= 0.95
    L, _ = orc.lindblad(prob, 1e-10, 1e-12)
    _within_statistics(g["mean"], g["se"], L, 403)


def test_removing_the_drive_restores_the_static_run():
    """qtm_set_drive with no terms gives bitwise the run of a context that never had them."""
    prob = S.jaynes_cummings_pulsed(ntraj=64)
    static = prob.with_(drive=[])
    a = gpu_run(static, 64, precision=Q.QTM_PREC_DF64, record=8)
    ctx = Q.qtm_create(prob, precision=Q.QTM_PREC_DF64, record_jumps=8)
    Q.qtm_set_drive(ctx, [])
    Q.qtm_run(ctx, 64, prob.seed)
    np.testing.assert_array_equal(Q.qtm_traj_expect(ctx), a["obs"])
    Q.qtm_destroy(ctx)


def test_drive_argument_errors():
    prob = S.jaynes_cummings_pulsed(ntraj=4)
    ctx = Q.qtm_create(prob.with_(drive=[]), precision=Q.QTM_PREC_C128)
    n = prob.dim
    bad = sp.csr_matrix(np.triu(np.ones((n, n))) * 1j)
    for terms, status in [([(bad, 1.0, 1.0, 0.0)], Q.QTM_ERR_ARG),                       # not Hermitian
                          ([(S.sigma_z(), 1.0, 1.0, 0.0)], Q.QTM_ERR_ARG),                 # wrong dimension
                          ([(prob.drive[0][0], np.nan, 1.0, 0.0)], Q.QTM_ERR_ARG),         # non-finite
                          ([(prob.drive[0][0], 1.0, 1.0, 0.0)] * 9, Q.QTM_ERR_ARG)]:       # more than 8
        with pytest.raises(Q.QtmError) as ei:
            Q.qtm_set_drive(ctx, terms)
        assert ei.value.status == status
    Q.qtm_destroy(ctx)
    tc = Q.qtm_create(prob.with_(drive=[]), precision=Q.QTM_PREC_BF16X6)
    with pytest.raises(Q.QtmError) as ei:
        Q.qtm_set_drive(tc, prob.drive)
    assert ei.value.status == Q.QTM_ERR_UNSUPPORTED
    Q.qtm_destroy(tc)
