"""Edge cases of the energy layout against the oracle's term-by-term sum on
the same (FP32-rounded) state.  The kernel groups terms into classes by the
flipped bits above an L2-sized chunk, visits each pair from one side, and
runs 4096-amplitude blocks of 16 amplitudes per thread; these cases reach
each branch of that: the smallest register (below one block), registers
around one block, registers split into classes (FP32 from 23 qubits, FP64
from 22), many terms on few qubits, many terms on one flip, flips inside a
thread's own amplitudes (the per-element path) and of the top qubit only,
repeated flips with other phases, identity and diagonal terms, and
Hamiltonians with no diagonal or no flipping term."""
import numpy as np
import pytest

from energy_tol import energy_error
from oracle import oracle as orc
from paper_2609_23664_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_23664_gb300 import quwarp as Q  # noqa: E402

# FP32 products and butterflies, double-float accumulation (the bound of the
# kernel-level energy test)
KERNEL_ENERGY_TOL = 4e-7


@pytest.fixture(scope="module")
def eng():
    e = Q.Engine(0)
    yield e
    e.close()


def edge_terms(rng, n, k, kind="mixed"):
    t = W.random_pauli_hamiltonian(rng, n, k)
    if kind == "diagonal":
        t["xmask"] = 0
        return t
    if kind == "one_flip":  # every term flips the same qubits, phases differ
        t["xmask"] = t[0]["xmask"] | 1
        return t
    if kind == "flipping":
        t["xmask"] |= 1 << int(rng.integers(0, n))
        return t
    for i in range(0, k, 7):
        t[i]["xmask"] = 0
    t[1]["xmask"] = 0
    t[1]["zmask"] = 0
    for i in range(3, k, 11):
        t[i]["xmask"] = int(rng.integers(1, 8)) & ((1 << n) - 1)
    for i in range(5, k, 13):
        t[i]["xmask"] = t[i - 1]["xmask"]
    for i in range(6, k, 17):
        t[i]["xmask"] = 1 << (n - 1)
    return t


def check(eng, mode, n, terms, seed):
    rng = np.random.default_rng(seed)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi *= 0.9 / np.linalg.norm(psi)
    if mode == W.MODE_SV_FP32:
        psi = psi.astype(np.complex64).astype(np.complex128)
    dt = torch.complex128 if mode == W.MODE_SV_FP64 else torch.complex64
    st = torch.tensor(psi, dtype=dt, device="cuda")
    e, nr = Q.sv_energy_dev(eng, mode, n, st.data_ptr(), terms)
    e_ref, n_ref, _ = orc.energy(n, psi, terms)
    if mode == W.MODE_SV_FP64:
        assert abs(nr - n_ref) <= 1e-13 * n_ref
        assert abs(e - e_ref) <= 1e-12 * max(1.0, abs(e_ref)), (e, e_ref)
    else:
        assert abs(nr - n_ref) <= 1e-6 * n_ref
        err = energy_error(e, e_ref, terms, n)
        assert err <= KERNEL_ENERGY_TOL, (e, e_ref, err)


@pytest.mark.parametrize("mode,n,k", [(W.MODE_SV_FP32, 5, 40), (W.MODE_SV_FP64, 5, 40),
                                      (W.MODE_SV_FP32, 12, 120), (W.MODE_SV_FP32, 13, 120),
                                      (W.MODE_SV_FP32, 14, 120), (W.MODE_SV_FP64, 12, 120),
                                      (W.MODE_SV_FP64, 13, 120), (W.MODE_SV_FP32, 9, 700),
                                      (W.MODE_SV_FP64, 8, 500)])
def test_register_sizes_and_term_counts(eng, mode, n, k):
    rng = np.random.default_rng(1000 + 7 * n + k + mode)
    check(eng, mode, n, edge_terms(rng, n, k), 2000 + n)


@pytest.mark.parametrize("mode,n", [(W.MODE_SV_FP32, 23), (W.MODE_SV_FP32, 25), (W.MODE_SV_FP64, 22),
                                    (W.MODE_SV_FP64, 23)])
def test_chunk_classes(eng, mode, n):
    rng = np.random.default_rng(3000 + n + mode)
    check(eng, mode, n, edge_terms(rng, n, 90), 4000 + n)


@pytest.mark.parametrize("kind", ["diagonal", "one_flip", "flipping"])
@pytest.mark.parametrize("mode", [W.MODE_SV_FP32, W.MODE_SV_FP64])
def test_hamiltonian_shapes(eng, mode, kind):
    n = 16
    rng = np.random.default_rng(5000 + mode + len(kind))
    check(eng, mode, n, edge_terms(rng, n, 150, kind), 6000 + len(kind))
