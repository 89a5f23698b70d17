"""qs_expect_z_noalloc: the reduction entry point for callers that must not allocate
device memory (hosts that give all device memory to their own pool before loading
plug-ins, loops that cannot take cudaMalloc's device synchronisation).

It is called through the C ABI and compared with the allocating entry points
qs_expect(QS_NORM) and qs_expect_pauli(type 0) on the same states, twice in a row.
The fixed scratch array keeps the previous call's partial sums, so the second call
of each pair uses a smaller state and a different batch: a wrong read of slots the
first call left behind would change its answer.  This file is collected last on
purpose.
"""
import pytest

gpu = pytest.mark.gpu

OBS_TOL = 1e-6     # the observable tolerance of the parity tests


def _noalloc(Q, torch, sim, code, mask):
    batch = sim.batch
    out = torch.full((2 * batch,), float("nan"), dtype=torch.float64, device=sim.state.device)
    stream = torch.cuda.current_stream().cuda_stream
    Q.qs_expect_z_noalloc(sim.state.data_ptr(), sim.n, code, batch, mask, out.data_ptr(), stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _check(sim, got, mask):
    from paper_2108_13410_gb300 import QS_NORM
    norm_ref = sim.expect(QS_NORM)
    z_ref = sim.expect_pauli(0, mask)
    for b in range(sim.batch):
        assert abs(got[2 * b] - norm_ref[b]) <= OBS_TOL
        assert abs(got[2 * b + 1] - z_ref[b]) <= OBS_TOL


@gpu
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_noalloc_matches_allocating_entry_points(dtype):
    import torch
    from paper_2108_13410_gb300 import Simulator
    from paper_2108_13410_gb300 import qsim as Q

    code = Q.QS_C64 if dtype == "c64" else Q.QS_C128
    # large: 18 qubits, batch 5 -> every one of the 304 partial-sum blocks per element
    big = Simulator(3, 2, form="gh", dtype=dtype, batch=5)
    big.init_plus()
    big.evolve([(0.2, 0.2), (0.6, 0.6), (1.2, 1.2), (0.9, 0.1), (0.1, 0.9)], [0.1, 0.3, 0.5, 0.7], 0.2, 2)
    # small: 8 qubits (2x2 unitary gauge), batch 2 -> one block per element
    small = Simulator(2, 2, form="ug", dtype=dtype, batch=2)
    small.init_plus()
    small.evolve([(0.4, 0.3), (1.1, 0.7)], [0.2, 0.5, 0.8], 0.3, 2)
    mask_big = sum(1 << q for q in (0, 1, 6, 8))
    mask_small = sum(1 << q for q in (1, 2, 5))
    for _ in range(2):
        got = _noalloc(Q, torch, big, code, mask_big)
        _check(big, got, mask_big)
        got = _noalloc(Q, torch, small, code, mask_small)
        _check(small, got, mask_small)
    # all-qubit mask on the large state, then the small state again
    full = (1 << big.n) - 1
    _check(big, _noalloc(Q, torch, big, code, full), full)
    _check(small, _noalloc(Q, torch, small, code, mask_small), mask_small)


@gpu
@pytest.mark.parametrize("case", ["batch", "zmask", "n_low", "n_high", "dtype", "null_state", "null_out"])
def test_noalloc_rejects_bad_arguments(case):
    import torch
    from paper_2108_13410_gb300 import qsim as Q

    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    args = dict(state=x.data_ptr(), n=3, dtype=Q.QS_C64, batch=1, mask=1, out=out.data_ptr())
    word = {"batch": "batch", "zmask": "zmask", "n_low": "n_qubits", "n_high": "n_qubits",
            "dtype": "dtype", "null_state": "null", "null_out": "null"}[case]
    if case == "batch":
        args["batch"] = Q.QS_NOALLOC_MAX_BATCH + 1
    elif case == "zmask":
        args["mask"] = 1 << 3
    elif case == "n_low":
        args["n"] = 0
    elif case == "n_high":
        args["n"] = 35
    elif case == "dtype":
        args["dtype"] = 7
    elif case == "null_state":
        args["state"] = None
    elif case == "null_out":
        args["out"] = None
    with pytest.raises(Q.QsError) as e:
        Q.qs_expect_z_noalloc(args["state"], args["n"], args["dtype"], args["batch"], args["mask"], args["out"], 0)
    assert e.value.status == 1 and word in str(e.value)
    # nothing was written
    assert torch.count_nonzero(out).item() == 0
