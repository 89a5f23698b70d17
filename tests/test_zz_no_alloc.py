"""qs_expect_z_noalloc: the reduction entry point for callers that must not allocate
device memory (graph-capture regions, hosts that pool all device memory, loops that
cannot afford cudaMalloc's device synchronisation).

It is called through the C ABI and compared with the allocating entry points
qs_expect(QS_NORM) and qs_expect_pauli(type 0) on the same states, twice in a row
(the fixed scratch array keeps the previous call's partial sums, so a second call
must not be affected by the first).  This file is collected last on purpose.
"""
import pytest

gpu = pytest.mark.gpu

OBS_TOL = 1e-6     # the observable tolerance of the parity tests


@gpu
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_noalloc_matches_allocating_entry_points(dtype):
    import torch
    from paper_2108_13410_gb300 import Simulator, QS_NORM
    from paper_2108_13410_gb300 import qsim as Q

    batch = 3
    sim = Simulator(3, 2, form="gh", dtype=dtype, batch=batch)
    sim.init_plus()
    sim.evolve([(0.2, 0.2), (0.6, 0.6), (1.2, 1.2)], [0.1, 0.3, 0.5, 0.7], 0.2, 2)
    masks = [sum(1 << q for q in (0, 1, 6, 8)), (1 << sim.n) - 1]
    out = torch.full((2 * batch,), float("nan"), dtype=torch.float64, device=sim.state.device)
    code = Q.QS_C64 if dtype == "c64" else Q.QS_C128
    stream = torch.cuda.current_stream().cuda_stream
    for mask in masks:
        norm_ref = sim.expect(QS_NORM)
        z_ref = sim.expect_pauli(0, mask)
        for _ in range(2):
            Q.qs_expect_z_noalloc(sim.state.data_ptr(), sim.n, code, batch, mask, out.data_ptr(), stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            for b in range(batch):
                assert abs(got[2 * b] - norm_ref[b]) <= OBS_TOL
                assert abs(got[2 * b + 1] - z_ref[b]) <= OBS_TOL


@gpu
def test_noalloc_rejects_oversized_batch():
    import torch
    from paper_2108_13410_gb300 import qsim as Q

    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(Q.QsError) as e:
        Q.qs_expect_z_noalloc(x.data_ptr(), 3, Q.QS_C64, 17, 1, out.data_ptr(), 0)
    assert e.value.status == 1 and "batch" in str(e.value)
