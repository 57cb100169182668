"""The allocation-free evaluation entry point (for callers that cannot call
cudaMalloc, e.g. code confined to a memory pool it does not own) gives the
same unsatisfied counts, SAT masks and losses as tsat_evaluate, on two calls
in a row through the C ABI, and its second call leaves the device's free
memory unchanged.  Collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300 import turbosat as ts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("N,batch", [(64, False), (256, True)])
def test_noalloc_matches_evaluate_twice(N, batch):
    insts = cnfgen.batch_ksat(3, 5, n_lo=150, n_hi=900) if batch else [cnfgen.planted_ksat(2000, 8400, 3, 3)]
    prob = ts.Problem([(i.n_vars, i.clause_ptr, i.lits) for i in insts])
    st = ts.State(prob, N)
    hp = ts.hparams(seed=9, norm=1, tau=1.3)
    ts.tsat_init(st.h, hp)
    I = prob.info["n_inst"]
    for call in range(2):
        ts.tsat_step(st.h, hp, 3, stop_on_sat=False)
        u_ref = torch.zeros(I * N, dtype=torch.int32, device="cuda")
        m_ref = torch.zeros(I * N // 32, dtype=torch.int32, device="cuda")
        l_ref = torch.zeros(I, dtype=torch.float32, device="cuda")
        ts.tsat_evaluate(st.h, hp, u_ref, m_ref, l_ref)
        bits = st.view("bits").clone()
        u = torch.full((I * N,), -7, dtype=torch.int32, device="cuda")
        m = torch.full((I * N // 32,), -7, dtype=torch.int32, device="cuda")
        loss = torch.full((I,), 123.0, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        ts.tsat_evaluate_bits_noalloc(prob.h, bits, N, hp.tau, u, m, loss)
        torch.cuda.synchronize()
        if call == 1:
            # after the first call (which may load the library's device code and
            # look up the array), a call takes no device memory at all
            assert torch.cuda.mem_get_info()[0] == free_before
        np.testing.assert_array_equal(u.cpu().numpy(), u_ref.cpu().numpy())
        np.testing.assert_array_equal(m.cpu().numpy(), m_ref.cpu().numpy())
        ref = l_ref.cpu().numpy()
        assert np.max(np.abs(loss.cpu().numpy() - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_noalloc_rejects_oversize():
    inst = cnfgen.planted_ksat(200, 800, 3, 1)
    prob = ts.Problem([(inst.n_vars, inst.clause_ptr, inst.lits)])
    # 1024 samples x 400 instances would need far more than the fixed array
    big = cnfgen.batch_ksat(400, 2, n_lo=20, n_hi=30, k_hi=3)
    bprob = ts.Problem([(i.n_vars, i.clause_ptr, i.lits) for i in big])
    bits = torch.zeros(bprob.info["n_vars"] * 32, dtype=torch.int32, device="cuda")
    u = torch.zeros(400 * 1024, dtype=torch.int32, device="cuda")
    m = torch.zeros(400 * 32, dtype=torch.int32, device="cuda")
    with pytest.raises(ts.TsatError) as e:
        ts.tsat_evaluate_bits_noalloc(bprob.h, bits, 1024, 1.0, u, m, None)
    assert e.value.status == -10
    del prob
