"""The non-allocating energy entry point (qw_sv_energy_noalloc_dev).

It exists for callers that cannot allocate device memory (device memory
owned by another allocator, latency-bound loops with a fixed memory
footprint that cannot afford cudaFree's synchronization).  This test calls
it through the C ABI twice in a row and checks each result against the
allocating entry point (qw_sv_energy_dev) on the same state, within the
tolerance the other energy tests use, at the edges of its fixed scratch
array: 26 qubits with 1024 terms spread over all eight term classes (every
block slot of the array used), registers below one 4096-amplitude block,
and an empty term list.  The file name makes pytest collect it last."""
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


def _terms(rng, n, n_terms, every_class):
    terms = W.random_pauli_hamiltonian(rng, n, n_terms)
    if n_terms:
        terms[0]["xmask"] = 0
    if every_class and n >= 15:
        # the top three qubits' flips cycle through all eight class patterns
        for k in range(n_terms):
            hi = np.uint64(k % 8) << np.uint64(n - 3)
            low = terms[k]["xmask"] & np.uint64((1 << (n - 3)) - 1)
            terms[k]["xmask"] = hi | low
    return terms


@pytest.mark.parametrize("mode,n,n_terms,every_class", [(W.MODE_SV_FP32, 17, 120, False),
                                                        (W.MODE_SV_FP64, 12, 40, False),
                                                        (W.MODE_SV_FP32, 26, 1024, True),
                                                        (W.MODE_SV_FP64, 5, 7, False),
                                                        (W.MODE_SV_FP32, 9, 30, False),
                                                        (W.MODE_SV_FP32, 14, 0, False)])
def test_noalloc_energy_matches_allocating_entry_point(mode, n, n_terms, every_class):
    eng = Q.Engine(0)
    rng = np.random.default_rng(900 + n)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for call in range(2):  # two calls in a row reuse the same scratch array
        st = _state(rng, n, mode)
        terms = _terms(rng, n, n_terms, every_class)
        Q.sv_energy_noalloc_dev(mode, n, st.data_ptr(), terms, out.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        e, nr = out.cpu().numpy()
        e_ref, n_ref = Q.sv_energy_dev(eng, mode, n, st.data_ptr(), terms)
        # the two add the same terms in a different order (their term classes
        # differ); the FP32 bound is the kernel bound of the parity tests
        if mode == W.MODE_SV_FP64:
            assert abs(e - e_ref) <= 1e-12 * max(1.0, abs(e_ref)), (call, e, e_ref)
        else:
            e_typ = float(np.sqrt(np.sum(terms["coef"] ** 2))) * 2.0 ** (-n / 2) if n_terms else 1.0
            assert abs(e - e_ref) <= 4e-7 * max(abs(e_ref), e_typ), (call, e, e_ref)
        tol = 1e-12 if mode == W.MODE_SV_FP64 else 1e-9
        assert abs(nr - n_ref) <= tol * n_ref, (call, nr, n_ref)
        if n_terms == 0:
            assert e == 0.0 and e_ref == 0.0
        del st
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
    with pytest.raises(Q.QuwarpError) as ei:  # below the 5-qubit padding: a malformed size
        Q.sv_energy_noalloc_dev(W.MODE_SV_FP32, 4, st.data_ptr(), too_many[:0], out.data_ptr())
    assert ei.value.status == -1  # QW_ERR_INVALID_ARG
