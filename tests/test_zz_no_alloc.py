"""The non-allocating energy entry point (qw_sv_energy_noalloc_dev).

It exists for callers that cannot allocate device memory (work issued during
a global-mode graph capture, memory owned by another allocator,
latency-bound loops that cannot afford cudaFree's synchronization).  This
test calls it through the C ABI twice in a row and checks each result
against the allocating entry point (qw_sv_energy_dev) on the same state,
within the tolerance the other energy tests use.  The file name makes
pytest collect it last."""
import numpy as np
import pytest

from paper_2609_23664_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2609_23664_gb300 import quwarp as Q  # noqa: E402


def _state(rng, n, mode):
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi *= 0.9 / np.linalg.norm(psi)
    dt = torch.complex128 if mode == W.MODE_SV_FP64 else torch.complex64
    return torch.tensor(psi, dtype=dt, device="cuda")


@pytest.mark.parametrize("mode,n,n_terms", [(W.MODE_SV_FP32, 17, 120), (W.MODE_SV_FP64, 12, 40)])
def test_noalloc_energy_matches_allocating_entry_point(mode, n, n_terms):
    eng = Q.Engine(0)
    rng = np.random.default_rng(900 + n)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for call in range(2):  # two calls in a row reuse the same scratch array
        st = _state(rng, n, mode)
        terms = W.random_pauli_hamiltonian(rng, n, n_terms)
        terms[0]["xmask"] = 0
        Q.sv_energy_noalloc_dev(mode, n, st.data_ptr(), terms, out.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        e, nr = out.cpu().numpy()
        e_ref, n_ref = Q.sv_energy_dev(eng, mode, n, st.data_ptr(), terms)
        tol = 1e-12 if mode == W.MODE_SV_FP64 else 1e-9
        assert abs(e - e_ref) <= tol * max(1.0, abs(e_ref)), (call, e, e_ref)
        assert abs(nr - n_ref) <= tol * n_ref, (call, nr, n_ref)
    eng.close()


def test_noalloc_rejects_sizes_beyond_the_scratch_array():
    st = torch.zeros(1 << 5, dtype=torch.complex64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    too_many = W.random_pauli_hamiltonian(np.random.default_rng(1), 5, 1025)
    with pytest.raises(Q.QuwarpError) as ei:
        Q.sv_energy_noalloc_dev(W.MODE_SV_FP32, 5, st.data_ptr(), too_many, out.data_ptr())
    assert ei.value.status == -3  # QW_ERR_BUDGET
    with pytest.raises(Q.QuwarpError) as ei:
        Q.sv_energy_noalloc_dev(W.MODE_SV_FP32, 27, st.data_ptr(), too_many[:3], out.data_ptr())
    assert ei.value.status == -3
