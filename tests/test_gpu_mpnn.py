"""Learned proposer on the GPU: forward and gradient against the FP64 oracle,
training decreases the loss, and the trained network beats random init."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mpnn
from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300 import turbosat as ts
from paper_2511_07737_b300.proposer import Proposer, compare, make_dataset
from tests.conftest import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)


def test_mpnn_forward_and_gradient_match_oracle():
    insts = [cnfgen.planted_ksat(300, 1150, 3, 2), cnfgen.planted_ksat(200, 3800, 5, 3),
             cnfgen.tiny_random(40, 120, 4, kmin=1, kmax=6)]
    prob = ts.Problem([(i.n_vars, i.clause_ptr, i.lits) for i in insts])
    pr = Proposer(seed=7)
    y = np.concatenate([i.planted for i in insts]).astype(np.uint8)
    ws = pr._ws(prob)
    logits = torch.empty(prob.info["n_vars"], device="cuda")
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros_like(pr.params)
    ts.tsat_mpnn_loss_grad(prob.h, pr.params, ws, torch.tensor(y, device="cuda"), logits, loss, grad)
    ts.tsat_mpnn_status(prob.h, ws)                          # every tensor-core layer's wait completed
    params = mpnn.bf16_round(pr.params.cpu().numpy())       # the kernels compute with BF16 weights
    g = mpnn.Graph([oracle.CNF(i.n_vars, i.clause_ptr, i.lits) for i in insts])
    l_ref, g_ref, lg_ref = mpnn.loss_and_grad(g, params, y)
    assert rel_err(logits.cpu().numpy(), lg_ref) < 1e-5
    assert abs(loss.item() - l_ref) < 1e-5 * abs(l_ref)
    assert rel_err(grad.cpu().numpy(), g_ref) < 1e-4


@pytest.mark.parametrize("name,gen", [
    # every forward layer at most 2,048 rows: the CUDA-core form of the layers
    ("n100", lambda: [cnfgen.planted_ksat(100, 426, 3, 8)]),
    # literal layer on CUDA cores (1,400 rows), clause layer on the tensor cores (2,982 rows)
    ("n700", lambda: [cnfgen.planted_ksat(700, 2982, 3, 9)]),
])
def test_mpnn_small_layers_match_oracle(name, gen):
    """Forward logits, loss and gradient on graphs whose layers are small
    enough for the CUDA-core form (a clause layer of at most 2,048 rows, a
    literal layer of at most 1,536), alone and mixed with tensor-core layers."""
    insts = gen()
    prob = ts.Problem([(i.n_vars, i.clause_ptr, i.lits) for i in insts])
    pr = Proposer(seed=13)
    y = np.concatenate([i.planted for i in insts]).astype(np.uint8)
    ws = pr._ws(prob)
    logits = torch.empty(prob.info["n_vars"], device="cuda")
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros_like(pr.params)
    ts.tsat_mpnn_loss_grad(prob.h, pr.params, ws, torch.tensor(y, device="cuda"), logits, loss, grad)
    ts.tsat_mpnn_status(prob.h, ws)
    params = mpnn.bf16_round(pr.params.cpu().numpy())
    g = mpnn.Graph([oracle.CNF(i.n_vars, i.clause_ptr, i.lits) for i in insts])
    l_ref, g_ref, lg_ref = mpnn.loss_and_grad(g, params, y)
    assert rel_err(logits.cpu().numpy(), lg_ref) < 1e-5
    assert abs(loss.item() - l_ref) < 1e-5 * abs(l_ref)
    assert rel_err(grad.cpu().numpy(), g_ref) < 1e-4
    # the forward alone (the proposal path) gives the same logits
    lg2 = torch.empty_like(logits)
    ts.tsat_mpnn_forward(prob.h, pr.params, ws, lg2)
    ts.tsat_mpnn_status(prob.h, ws)
    assert rel_err(lg2.cpu().numpy(), lg_ref) < 1e-5


def test_mpnn_matches_oracle_when_blocks_loop_over_tiles():
    # 66,000 literal rows and 156,000 clause rows: more 128-row tiles than the
    # dense layers launch blocks (148 x 3), so every block loops over tiles,
    # and the weight-gradient blocks each reduce dozens of 32-row tiles
    insts = [cnfgen.planted_ksat(30000, 126000, 3, 5), cnfgen.planted_ksat(3000, 30000, 5, 6)]
    prob = ts.Problem([(i.n_vars, i.clause_ptr, i.lits) for i in insts])
    pr = Proposer(seed=11)
    y = np.concatenate([i.planted for i in insts]).astype(np.uint8)
    ws = pr._ws(prob)
    logits = torch.empty(prob.info["n_vars"], device="cuda")
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros_like(pr.params)
    ts.tsat_mpnn_loss_grad(prob.h, pr.params, ws, torch.tensor(y, device="cuda"), logits, loss, grad)
    torch.cuda.synchronize()
    params = mpnn.bf16_round(pr.params.cpu().numpy())
    g = mpnn.Graph([oracle.CNF(i.n_vars, i.clause_ptr, i.lits) for i in insts])
    l_ref, g_ref, lg_ref = mpnn.loss_and_grad(g, params, y)
    assert rel_err(logits.cpu().numpy(), lg_ref) < 1e-5
    assert abs(loss.item() - l_ref) < 1e-5 * abs(l_ref)
    assert rel_err(grad.cpu().numpy(), g_ref) < 1e-4


def test_training_lowers_loss_and_learned_init_beats_random():
    # solver settings and ratios where the gradient solver finds models within
    # the step cap (3-SAT at 0.9x, 5-SAT at 0.5x, 4-SAT at 0.6x of threshold)
    hp = ts.hparams(seed=3, norm=ts.NORM_ABSMEAN, tau=2.0, lr0=0.5)
    train = (cnfgen.batch_ksat(64, 101, n_lo=200, n_hi=600, ks=[3], ratio_scale=0.9)
             + cnfgen.batch_ksat(48, 102, n_lo=200, n_hi=500, ks=[5], ratio_scale=0.5))
    data, dropped = make_dataset(train, N=32, hp=hp, max_steps=1000)
    assert len(data) >= 60, (len(data), dropped)
    pr = Proposer(seed=1)
    hist = pr.fit(data, epochs=8, batch=16, lr=3e-3)
    assert np.mean(hist[-6:]) < np.mean(hist[:6])
    test = cnfgen.batch_ksat(48, 202, n_lo=300, n_hi=600, ks=[4], ratio_scale=0.6)
    # the proposal alone: fewer unsatisfied clauses than random init at step 0
    prob = ts.Problem([(i.n_vars, i.clause_ptr, i.lits) for i in test])
    lg = pr.logits(prob)
    counts = []
    for logits in (None, lg):
        st = ts.State(prob, 32)
        ts.tsat_init(st.h, hp, logits, 1.0)
        unsat = torch.zeros(len(test) * 32, dtype=torch.int32, device="cuda")
        sm = torch.zeros(len(test), dtype=torch.int32, device="cuda")
        ts.tsat_evaluate(st.h, hp, unsat, sm)
        counts.append(unsat.float().mean().item())
    assert counts[1] < 0.9 * counts[0], counts
    res = compare(test, pr, N=32, hp=hp, max_steps=1000)
    assert res["learned"]["solved"] >= res["random"]["solved"] - 2, res
    if res.get("matched_k", 0) >= 10:
        m = res["matched_median_steps"]
        assert m["learned"] <= m["random"], res


def test_mpnn_forward_closed_form_on_the_hand_sized_graph():
    """The selector weights (exact in BF16) of the oracle's composition pin:
    the kernels' logits equal the closed form computed from the clause lists."""
    from tests.test_oracle_mpnn import _selector_logits_by_hand, _selector_params
    clauses = [[(0, 0), (1, 1)], [(0, 0), (1, 0), (2, 0)], [(0, 0), (2, 1), (3, 0)], [(0, 1), (3, 0)]]
    ptr = np.array([0, 2, 5, 8, 10], np.int64)
    lits = np.array([1, -2, 1, 2, 3, 1, -3, 4, -1, 4], np.int32)
    prob = ts.Problem([(4, ptr, lits)])
    params = torch.tensor(_selector_params(), dtype=torch.float32, device="cuda")
    ws = torch.empty((ts.tsat_mpnn_workspace_bytes(prob.h) + 7) // 8, dtype=torch.int64, device="cuda")
    logits = torch.empty(4, device="cuda")
    ts.tsat_mpnn_forward(prob.h, params, ws, logits)
    torch.cuda.synchronize()
    want = _selector_logits_by_hand(4, clauses)
    assert rel_err(logits.cpu().numpy(), want) < 1e-5


def test_mpnn_calls_check_their_workspace():
    """A workspace that is too small or not 256-byte aligned is an argument
    error (no launch); a good one reports every tensor-core wait completed."""
    inst = cnfgen.planted_ksat(300, 1150, 3, 2)
    prob = ts.Problem([(inst.n_vars, inst.clause_ptr, inst.lits)])
    pr = Proposer(seed=7)
    ws = pr._ws(prob)
    logits = torch.empty(prob.info["n_vars"], device="cuda")
    with pytest.raises(ts.TsatError) as e:
        ts.tsat_mpnn_forward(prob.h, pr.params, ws[: ws.numel() // 2], logits)
    assert e.value.status == -4                  # TSAT_EWS
    big = torch.empty(ws.numel() + 64, dtype=torch.int64, device="cuda")
    shifted = big.view(torch.uint8)[16:16 + ws.numel() * 8]   # large enough, 16 bytes past an aligned start
    with pytest.raises(ts.TsatError) as e:
        ts.tsat_mpnn_forward(prob.h, pr.params, shifted, logits)
    assert e.value.status == -1 and "aligned" in str(e.value)   # TSAT_EINVAL
    with pytest.raises(ts.TsatError) as e:
        ts.tsat_mpnn_status(prob.h, shifted)
    assert e.value.status == -1
    ts.tsat_mpnn_forward(prob.h, pr.params, ws, logits)
    ts.tsat_mpnn_status(prob.h, ws)
    assert torch.isfinite(logits).all()


def test_forward_graph_replay_equals_direct_forward():
    """The forward replayed as a captured graph (second and later calls with the
    same buffers) gives the logits of a direct run bit for bit, also after the
    parameters change in place (the graph reads them when it runs)."""
    inst = cnfgen.planted_ksat(300, 1150, 3, 2)
    prob = ts.Problem([(inst.n_vars, inst.clause_ptr, inst.lits)])
    pr = Proposer(seed=7)
    ws = pr._ws(prob)
    lg = torch.empty(prob.info["n_vars"], device="cuda")

    def direct():
        ws2 = pr._ws(prob)   # other buffers: a direct run
        out = torch.empty_like(lg)
        ts.tsat_mpnn_forward(prob.h, pr.params, ws2, out)
        ts.tsat_mpnn_status(prob.h, ws2)
        return out.cpu().numpy()

    ref = direct()
    for _ in range(3):                  # direct, capture, replay
        lg.fill_(float("nan"))
        ts.tsat_mpnn_forward(prob.h, pr.params, ws, lg)
        ts.tsat_mpnn_status(prob.h, ws)
        np.testing.assert_array_equal(lg.cpu().numpy(), ref)
    with torch.no_grad():
        pr.params.mul_(0.5)
    ref2 = direct()
    assert not np.array_equal(ref, ref2)
    ts.tsat_mpnn_forward(prob.h, pr.params, ws, lg)   # the cached graph was dropped by the direct run
    ts.tsat_mpnn_forward(prob.h, pr.params, ws, lg)
    ts.tsat_mpnn_status(prob.h, ws)
    np.testing.assert_array_equal(lg.cpu().numpy(), ref2)
