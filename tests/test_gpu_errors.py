"""Argument validation of the C ABI: every bad call returns an error status and a
message, and leaves the simulator usable."""
import numpy as np
import pytest

gpu = pytest.mark.gpu


@gpu
def test_bad_arguments_are_rejected():
    import torch
    from paper_2108_13410_gb300 import qsim as Q
    for args in [(0, 3), (3, 0)]:
        with pytest.raises(Q.QsError) as e:
            Q.qs_create(*args)
        assert e.value.status == 1
    with pytest.raises(Q.QsError):
        Q.qs_create(6, 6)                        # 108 qubits
    with pytest.raises(Q.QsError):
        Q.qs_create(3, 3, 0, 0, 0, 70000)        # batch too large
    with pytest.raises(Q.QsError):
        Q.qs_create(3, 3, 7)                     # bad boundary
    h = Q.qs_create(3, 2)
    n = Q.qs_num_qubits(h)
    buf = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    with pytest.raises(Q.QsError):
        Q.qs_bind_state(h, 0, buf.data_ptr(), 16)          # too small
    with pytest.raises(Q.QsError):
        Q.qs_bind_state(h, 0, buf.data_ptr() + 8, buf.numel() * 8)   # misaligned
    with pytest.raises(Q.QsError):
        Q.qs_bind_state(h, 2, buf.data_ptr(), buf.numel() * 8)       # bad slot
    Q.qs_bind_state(h, 0, buf.data_ptr(), buf.numel() * 8)
    Q.qs_init_plus(h)
    with pytest.raises(Q.QsError):
        Q.qs_expect(h, 99)
    with pytest.raises(Q.QsError):
        Q.qs_expect(h, 3, n)                     # QS_X index out of range
    with pytest.raises(Q.QsError):
        Q.qs_expect_pauli(h, 0, 1 << n)          # mask beyond the qubits
    with pytest.raises(Q.QsError):
        Q.qs_set_option(h, 1, -1)
    with pytest.raises(Q.QsError):
        Q.qs_adjoint_grad(h, [(0.6, 0.6)], [0.5], 0.1, 2)    # no work state bound
    host = torch.empty(3, dtype=torch.complex64)
    with pytest.raises(Q.QsError):
        Q.qs_upload_state(h, host.data_ptr(), 24)
    with pytest.raises(Q.QsError):
        Q.qs_init_toric(h, 0)                    # gauge-Higgs form
    # still usable
    Q.qs_evolve(h, [(0.6, 0.6)], [0.2, 0.4], 0.1, 2)
    norm = Q.qs_expect(h, 0)[0]
    assert abs(norm - 1.0) < 1e-5
    assert "" != Q.qs_last_error(h)
    Q.qs_destroy(h)
