"""Seeded, synthetic inputs for the Monte Carlo wave-function (quantum trajectory) method.

This module builds the *inputs* of the method only: the system Hamiltonian H, the
collapse operators C_n, the observables A_k, the initial state psi0 and the output
time grid, for every workload the library is measured or tested on.  It contains
none of the method's arithmetic (no effective Hamiltonian, no integration, no jump
logic), so both the CUDA path and the CPU oracle can consume the same arrays
without sharing any computation.

Conventions (the paper prints none for these systems, so they are fixed here):

* hbar = 1 (the paper's unitary example, Sec. 4.1, stores its matrices with hbar = 1).
* Two-level systems: basis index 0 = |e> (excited / "up"), index 1 = |g> (ground /
  "down").  sigma_- = |g><e| = [[0,0],[1,0]], sigma_z = diag(1,-1), matching the
  Pauli matrices printed in Sec. 4.1.
* Tensor products are ordered as written (cavity (x) qubit, site 0 first), i.e. the
  state index is the mixed-radix number whose most significant digit is the first
  factor, the same order as the paper's ``tensor(d1, eye2)`` in Sec. 4.3.
* All operators are returned as ``scipy.sparse.csr_matrix`` of complex128 with
  sorted column indices and explicit zeros removed.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np
import scipy.linalg
import scipy.sparse as sp

__all__ = [
    "Problem", "destroy", "sigma_minus", "sigma_z", "sigma_x", "sigma_y", "kron",
    "two_level_driven", "jaynes_cummings_driven", "dense_random", "ising_chain",
    "ising_batch", "learned_proposal_system", "paper_unitary", "paper_trilinear",
    "paper_jaynes_cummings", "paper_photon_birth_death", "fock_decay", "purcell_qubit", "by_name",
]


@dataclasses.dataclass
class Problem:
    """One open-system workload: the paper's problem statement (Sec. 3, mpi_main).

    ``H``: system Hamiltonian (Hermitian), ``C``: collapse operators in channel
    order, ``A``: observables, ``psi0``: initial state, ``t``: strictly increasing
    output times (``t[0]`` is the start time), ``rtol``/``atol``: integrator
    tolerances, ``ntraj``/``seed``: ensemble size and random-stream key.
    ``dense``: the operators are dense matrices (pass them in dense format).
    ``drive``: time-dependent terms (H_k, a_k, omega_k, phi_k) adding
    a_k cos(omega_k t + phi_k) H_k to H (each H_k Hermitian).
    """

    name: str
    H: sp.csr_matrix
    C: List[sp.csr_matrix]
    A: List[sp.csr_matrix]
    psi0: np.ndarray
    t: np.ndarray
    rtol: float = 1e-8
    atol: float = 1e-10
    ntraj: int = 1000
    seed: int = 1
    dense: bool = False
    max_steps: int = 1_000_000
    obs_names: Optional[List[str]] = None
    drive: List[Tuple[sp.csr_matrix, float, float, float]] = dataclasses.field(default_factory=list)

    @property
    def dim(self) -> int:
        return int(self.H.shape[0])

    def with_(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# ----------------------------------------------------------------------------
# elementary operators
# ----------------------------------------------------------------------------

def _csr(m) -> sp.csr_matrix:
    out = sp.csr_matrix(m, dtype=np.complex128)
    out.eliminate_zeros()
    out.sort_indices()
    return out


def destroy(n: int) -> sp.csr_matrix:
    """Truncated bosonic annihilation operator a|k> = sqrt(k)|k-1>, k < n."""
    d = np.sqrt(np.arange(1, n, dtype=np.float64))
    return _csr(sp.diags(d, 1, shape=(n, n)))


def sigma_minus() -> sp.csr_matrix:
    """|g><e| with |e> = index 0 and |g> = index 1."""
    return _csr(np.array([[0, 0], [1, 0]], dtype=np.complex128))


def sigma_z() -> sp.csr_matrix:
    return _csr(np.diag([1.0, -1.0]).astype(np.complex128))


def sigma_x() -> sp.csr_matrix:
    return _csr(np.array([[0, 1], [1, 0]], dtype=np.complex128))


def sigma_y() -> sp.csr_matrix:
    return _csr(np.array([[0, -1j], [1j, 0]], dtype=np.complex128))


def eye(n: int) -> sp.csr_matrix:
    return _csr(sp.identity(n, dtype=np.complex128))


def kron(*ops) -> sp.csr_matrix:
    out = ops[0]
    for o in ops[1:]:
        out = sp.kron(out, o, format="csr")
    return _csr(out)


def dag(op) -> sp.csr_matrix:
    return _csr(op.conj().T)


def basis(n: int, k: int) -> np.ndarray:
    v = np.zeros(n, dtype=np.complex128)
    v[k] = 1.0
    return v


def coherent(n: int, alpha: complex) -> np.ndarray:
    """Truncated coherent state D(alpha)|0> with the displacement exponentiated
    on the n-level space (the construction of the paper's trilinear listing,
    Sec. 4.2: exp(alpha a^dag - conj(alpha) a) applied to the vacuum)."""
    a = destroy(n).toarray()
    gen = alpha * a.conj().T - np.conj(alpha) * a
    return scipy.linalg.expm(gen) @ basis(n, 0)


# ----------------------------------------------------------------------------
# measured / tested workloads
# ----------------------------------------------------------------------------

def two_level_driven(ntraj: int = 1000, seed: int = 1, n_t: int = 201, t_end: float = 50.0,
                     delta: float = 0.0, omega: float = 1.0, gamma: float = 0.1,
                     extra_sigma_y: bool = False) -> Problem:
    """Driven damped two-level atom, N = 2.

    H = Delta sigma_+ sigma_- + (Omega/2)(sigma_+ + sigma_-), C = sqrt(gamma) sigma_-,
    psi0 = |g>, observables sigma_+ sigma_- and sigma_x (optionally sigma_y).
    """
    sm = sigma_minus()
    spl = dag(sm)
    H = _csr(delta * (spl @ sm) + 0.5 * omega * (spl + sm))
    A = [_csr(spl @ sm), sigma_x()]
    names = ["sigma+sigma-", "sigma_x"]
    if extra_sigma_y:
        A.append(sigma_y())
        names.append("sigma_y")
    return Problem("two_level_driven", H, [_csr(math.sqrt(gamma) * sm)], A, basis(2, 1),
                   np.linspace(0.0, t_end, n_t), 1e-8, 1e-10, ntraj, seed, obs_names=names)


def jaynes_cummings_driven(ntraj: int = 20000, seed: int = 1, n_fock: int = 30, n_t: int = 401,
                           t_end: float = 40.0, g: float = 1.0, E: float = 0.5,
                           kappa: float = 0.2, gamma: float = 0.05) -> Problem:
    """Damped, driven Jaynes-Cummings model in the rotating frame (omega_c = omega_a = 0).

    Cavity Fock cutoff ``n_fock`` (x) qubit, N = 2 n_fock.
    H = g (a^dag sigma_- + a sigma_+) + E (a + a^dag), C1 = sqrt(kappa) a, C2 = sqrt(gamma) sigma_-,
    psi0 = |0> (x) |e>, observables a^dag a and sigma_+ sigma_-.
    """
    a = kron(destroy(n_fock), eye(2))
    sm = kron(eye(n_fock), sigma_minus())
    H = _csr(g * (dag(a) @ sm + a @ dag(sm)) + E * (a + dag(a)))
    C = [_csr(math.sqrt(kappa) * a), _csr(math.sqrt(gamma) * sm)]
    A = [_csr(dag(a) @ a), _csr(dag(sm) @ sm)]
    psi0 = np.kron(basis(n_fock, 0), basis(2, 0))
    return Problem("jaynes_cummings_driven", H, C, A, psi0, np.linspace(0.0, t_end, n_t),
                   1e-8, 1e-10, ntraj, seed, obs_names=["a^dag a", "sigma+sigma-"])


def dense_random(ntraj: int = 20000, seed: int = 1, N: int = 256, n_c: int = 4,
                 op_seed: int = 3, n_t: int = 101, t_end: float = 10.0,
                 c_norm: float = 0.3) -> Problem:
    """Dense random open system.

    H = (G + G^dag)/sqrt(2N) with G iid complex normal, E|g|^2 = 1 (GUE, entry
    variance 1/N); C_n = G_n * c_norm / ||G_n||_2 with G_n complex Ginibre;
    psi0 a normalised complex normal vector; observable diag(0..N-1)/N.
    Draw order from ``numpy.random.default_rng(op_seed)``: G, G_0..G_{n_c-1}, psi0.
    """
    rng = np.random.default_rng(op_seed)

    def ginibre():
        return (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) / math.sqrt(2.0)

    G = ginibre()
    H = (G + G.conj().T) / math.sqrt(2.0 * N)
    C = []
    for _ in range(n_c):
        Gn = ginibre()
        C.append(Gn * (c_norm / np.linalg.norm(Gn, 2)))
    psi0 = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    psi0 = psi0 / np.linalg.norm(psi0)
    A = [np.diag(np.arange(N, dtype=np.float64) / N).astype(np.complex128)]
    return Problem("dense_random", _csr(H), [_csr(c) for c in C], [_csr(x) for x in A], psi0,
                   np.linspace(0.0, t_end, n_t), 1e-8, 1e-10, ntraj, seed, dense=True,
                   obs_names=["diag(n)/N"])


ISING_TRAJ = {6: 50000, 7: 20000, 8: 10000, 9: 5000, 10: 2000}


def ising_chain(L: int, ntraj: Optional[int] = None, seed: int = 7, J: float = 1.0, h: float = 0.7,
                g_decay: float = 0.05, g_dephase: float = 0.02, n_t: int = 201,
                t_end: float = 20.0) -> Problem:
    """Open transverse-field Ising chain with L spins (N = 2^L), open boundaries.

    H = -J sum_i sz_i sz_{i+1} - h sum_i sx_i; channels ordered
    [sqrt(g_decay) s-_0 .. s-_{L-1}, sqrt(g_dephase) sz_0 .. sz_{L-1}];
    psi0 = all spins up (index 0); observables sz_i.  Site 0 is the most
    significant bit of the state index.
    """
    def site(op, i):
        return kron(*[op if j == i else eye(2) for j in range(L)])

    sz = [site(sigma_z(), i) for i in range(L)]
    sx = [site(sigma_x(), i) for i in range(L)]
    sm = [site(sigma_minus(), i) for i in range(L)]
    H = sp.csr_matrix((2 ** L, 2 ** L), dtype=np.complex128)
    for i in range(L - 1):
        H = H - J * (sz[i] @ sz[i + 1])
    for i in range(L):
        H = H - h * sx[i]
    C = [_csr(math.sqrt(g_decay) * s) for s in sm] + [_csr(math.sqrt(g_dephase) * s) for s in sz]
    if ntraj is None:
        ntraj = ISING_TRAJ.get(L, 2000)
    return Problem(f"ising_L{L}", _csr(H), C, [_csr(s) for s in sz], basis(2 ** L, 0),
                   np.linspace(0.0, t_end, n_t), 1e-8, 1e-10, ntraj, seed,
                   obs_names=[f"sz_{i}" for i in range(L)])


def ising_batch(Ls=(6, 7, 8, 9, 10)) -> List[Problem]:
    return [ising_chain(L) for L in Ls]


def driven_dephasing_qubit(ntraj: int = 500, seed: int = 1, a: float = 1.3, omega: float = 2.0,
                           phi: float = 0.4, gamma: float = 0.1, n_t: int = 101,
                           t_end: float = 10.0) -> Problem:
    """Time-dependent Hamiltonian with a closed form: H(t) = a cos(omega t + phi) sigma_z
    (the constant part of H is zero), dephasing C = sqrt(gamma) sigma_z, psi0 =
    |+> = (|0> + |1>)/sqrt 2, observables sigma_x and sigma_y.  With F(t) = the
    integral of the coefficient, a trajectory with N(t) jumps by time t has
    <sigma_x> = (-1)^N cos 2F and <sigma_y> = (-1)^N sin 2F; the ensemble mean of
    <sigma_x> is exp(-2 gamma t) cos 2F."""
    H0 = sp.csr_matrix((2, 2), dtype=np.complex128)
    psi0 = np.array([1.0, 1.0], dtype=np.complex128) / math.sqrt(2.0)
    return Problem("driven_dephasing_qubit", H0, [_csr(math.sqrt(gamma) * sigma_z())],
                   [sigma_x(), sigma_y()], psi0, np.linspace(0.0, t_end, n_t), 1e-8, 1e-10, ntraj, seed,
                   obs_names=["sigma_x", "sigma_y"], drive=[(sigma_z(), a, omega, phi)])


def jaynes_cummings_pulsed(ntraj: int = 2000, seed: int = 1, n_fock: int = 30, n_t: int = 201,
                           t_end: float = 20.0, g: float = 1.0, E: float = 0.8, omega: float = 0.7,
                           kappa: float = 0.2, gamma: float = 0.05) -> Problem:
    """The damped Jaynes-Cummings system with a modulated cavity drive instead of a
    constant one: H(t) = g (a^dag sigma_- + a sigma_+) + E cos(omega t) (a + a^dag),
    C = {sqrt(kappa) a, sqrt(gamma) sigma_-}, psi0 = |0> (x) |e>, observables
    a^dag a and sigma_+ sigma_-."""
    base = jaynes_cummings_driven(ntraj=ntraj, seed=seed, n_fock=n_fock, n_t=n_t, t_end=t_end, g=g, E=0.0,
                                  kappa=kappa, gamma=gamma)
    a = kron(destroy(n_fock), eye(2))
    return base.with_(name="jaynes_cummings_pulsed", drive=[(_csr(a + dag(a)), E, omega, 0.0)])


def learned_proposal_system(ntraj: int = 200000, seed: int = 1) -> Problem:
    """The Jaynes-Cummings system above at the ensemble size of the learned-proposal study."""
    return jaynes_cummings_driven(ntraj=ntraj, seed=seed).with_(name="learned_proposal_jc")


# ----------------------------------------------------------------------------
# the paper's own examples (Sec. 4)
# ----------------------------------------------------------------------------

def paper_unitary(ntraj: int = 1000, seed: int = 1, n_t: int = 101) -> Problem:
    """Sec. 4.1: H = (2 pi/10) sigma_x, C_0 = 0.05 sigma_x, E_0 = sigma_z, psi0 = |0>, t in [0, 10].

    Here |0> is basis index 0 (the paper's alpha = [1, 0]) and sigma_z = diag(1, -1).
    """
    H = _csr((2.0 * math.pi / 10.0) * sigma_x())
    return Problem("paper_unitary", H, [_csr(0.05 * sigma_x())], [sigma_z()], basis(2, 0),
                   np.linspace(0.0, 10.0, n_t), 1e-8, 1e-10, ntraj, seed, obs_names=["sigma_z"])


def paper_trilinear(ntraj: int = 1000, seed: int = 1, n_modes=(8, 8, 8), n_t: int = 100,
                    K: float = 1.0, gammas=(0.1, 0.1, 0.4), alpha: float = math.sqrt(3.0)) -> Problem:
    """Sec. 4.2: optical parametric amplifier H = i K (a b^dag c^dag - a^dag b c),
    c_i = sqrt(2 gamma_i) a_i, psi0 = |alpha>_a |0>_b |0>_c, observables n0, n1, n2, t in [0, 4]."""
    n0, n1, n2 = n_modes
    a0 = kron(destroy(n0), eye(n1), eye(n2))
    a1 = kron(eye(n0), destroy(n1), eye(n2))
    a2 = kron(eye(n0), eye(n1), destroy(n2))
    H = _csr(1j * K * (a0 @ dag(a1) @ dag(a2) - dag(a0) @ a1 @ a2))
    C = [_csr(math.sqrt(2.0 * g) * x) for g, x in zip(gammas, (a0, a1, a2))]
    A = [_csr(dag(x) @ x) for x in (a0, a1, a2)]
    psi0 = np.kron(np.kron(coherent(n0, alpha), basis(n1, 0)), basis(n2, 0))
    return Problem("paper_trilinear", H, C, A, psi0, np.linspace(0.0, 4.0, n_t), 1e-8, 1e-10,
                   ntraj, seed, obs_names=["n0", "n1", "n2"])


def paper_jaynes_cummings(n_fock: int = 40, g: float = 1.0, delta: float = -0.1, alpha: float = 4.0,
                          n_t: int = 600, t_end: float = 35.0) -> Problem:
    """Sec. 4.3: closed Jaynes-Cummings model, one trajectory, no collapse operators.

    a = d_N (x) I_2, b = I_N (x) sigma_-, H = Delta a^dag a + g (a^dag b + a b^dag),
    psi0 = coherent(alpha) (x) |1> (qubit basis index 1), observable b^dag b.
    """
    a = kron(destroy(n_fock), eye(2))
    b = kron(eye(n_fock), sigma_minus())
    H = _csr(delta * (dag(a) @ a) + g * (dag(a) @ b + a @ dag(b)))
    psi0 = np.kron(coherent(n_fock, alpha), basis(2, 1))
    return Problem("paper_jaynes_cummings", H, [], [_csr(dag(b) @ b)], psi0,
                   np.linspace(0.0, t_end, n_t), 1e-8, 1e-10, 1, 1, obs_names=["b^dag b"])


def paper_photon_birth_death(ntraj: int = 1000, seed: int = 1, N: int = 5, n_th: float = 0.063,
                             kappa: float = 1.0 / 0.129, n_t: int = 101, t_end: float = 1.0) -> Problem:
    """Sec. 4.4: H = a^dag a, psi0 = |1>, c_0 = sqrt(kappa (1 + n_th)) a, c_1 = sqrt(kappa n_th) a^dag.

    The paper calls n_th "t" (the thermal occupation of the environment)."""
    a = destroy(N)
    C = [_csr(math.sqrt(kappa * (1.0 + n_th)) * a), _csr(math.sqrt(kappa * n_th) * dag(a))]
    return Problem("paper_photon_birth_death", _csr(dag(a) @ a), C, [_csr(dag(a) @ a)],
                   basis(N, 1), np.linspace(0.0, t_end, n_t), 1e-8, 1e-10, ntraj, seed,
                   obs_names=["a^dag a"])


def fock_decay(n0: int = 3, n_fock: int = 6, kappa: float = 0.5, omega: float = 1.0,
               ntraj: int = 200, seed: int = 5, n_t: int = 81, t_end: float = 8.0) -> Problem:
    """Empty-cavity decay of a Fock state: H = omega a^dag a, C = sqrt(kappa) a, psi0 = |n0>."""
    a = destroy(n_fock)
    return Problem("fock_decay", _csr(omega * (dag(a) @ a)), [_csr(math.sqrt(kappa) * a)],
                   [_csr(dag(a) @ a)], basis(n_fock, n0), np.linspace(0.0, t_end, n_t), 1e-8, 1e-10,
                   ntraj, seed, obs_names=["a^dag a"])


def purcell_qubit(ntraj: int = 2000, seed: int = 1, n_fock: int = 5, g: float = 5.0, kappa: float = 200.0,
                  gamma: float = 0.05, omega: float = 0.5, n_t: int = 201, t_end: float = 20.0) -> Problem:
    """A stiff system: a driven qubit coupled to a strongly damped cavity (Purcell regime).

    a = d_N (x) I_2, b = I_N (x) sigma_-, H = g (a^dag b + a b^dag) + (omega / 2)(b + b^dag),
    C = {sqrt(kappa) a, sqrt(gamma) b}, psi0 = |0> (x) |e>, observables b^dag b and a^dag a.
    The cavity decays at kappa = 200 while the qubit relaxes through it at the Purcell
    rate 4 g^2 / kappa = 0.5: the rates of H_eff span more than two decades, so an
    explicit integrator's step is set by stability (h ~ 3.3 / (kappa n / 2)) rather
    than by accuracy (the setting of Sec. 2.1 where the paper switches ZVODE to BDF).
    """
    a = kron(destroy(n_fock), eye(2))
    b = kron(eye(n_fock), sigma_minus())
    H = _csr(g * (dag(a) @ b + a @ dag(b)) + 0.5 * omega * (b + dag(b)))
    C = [_csr(math.sqrt(kappa) * a), _csr(math.sqrt(gamma) * b)]
    A = [_csr(dag(b) @ b), _csr(dag(a) @ a)]
    psi0 = np.kron(basis(n_fock, 0), basis(2, 0))
    return Problem("purcell_qubit", H, C, A, psi0, np.linspace(0.0, t_end, n_t), 1e-8, 1e-10, ntraj, seed,
                   obs_names=["b^dag b", "a^dag a"])


def by_name(name: str, **kw) -> Problem:
    table = {
        "two_level_driven": two_level_driven,
        "jaynes_cummings_driven": jaynes_cummings_driven,
        "dense_random": dense_random,
        "learned_proposal_jc": learned_proposal_system,
        "paper_unitary": paper_unitary,
        "paper_trilinear": paper_trilinear,
        "paper_jaynes_cummings": paper_jaynes_cummings,
        "paper_photon_birth_death": paper_photon_birth_death,
        "fock_decay": fock_decay,
        "driven_dephasing_qubit": driven_dephasing_qubit,
        "jaynes_cummings_pulsed": jaynes_cummings_pulsed,
        "purcell_qubit": purcell_qubit,
    }
    if name.startswith("ising_L"):
        return ising_chain(int(name[len("ising_L"):]), **kw)
    return table[name](**kw)
