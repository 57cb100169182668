"""SatObjective (torch.autograd.Function over the C ABI) against the oracle,
finite differences, and the library's own fused AdamW step."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_07737_b300 import cnfgen
from paper_2511_07737_b300 import turbosat as ts
from paper_2511_07737_b300.autograd import SatObjective
from tests.conftest import rel_err
from tests.gpu_util import TOL_F32, assert_adamw_z, make, snapshot

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("norm", [0, 1, 2])
def test_autograd_gradient_matches_oracle(norm):
    inst = cnfgen.planted_ksat(700, 2982, 3, 31)
    prob, st, cnfs = make([inst], 64)
    hp = ts.hparams(seed=3, norm=norm, tau=1.2)
    g = torch.Generator(device="cuda").manual_seed(2)
    z = (torch.randn(700, 64, device="cuda", generator=g) + 0.6).requires_grad_(True)
    loss, S = SatObjective.apply(z, st, hp, 0)
    (2.5 * loss).backward()
    torch.cuda.synchronize()
    zc = z.detach().cpu().numpy()
    nu = st.view("nu").cpu().numpy()
    X = oracle.binarize_f32(zc, nu, 0)
    S_ref, L_ref, G, _ = oracle.objective(cnfs[0], X=X, tau=1.2)
    gref = 2.5 * oracle.normalize_backward(zc.astype(np.float64), nu.astype(np.float64), G, norm)
    assert abs(loss.item() - L_ref) < TOL_F32 * abs(L_ref)
    assert rel_err(S.cpu().numpy(), S_ref) < TOL_F32
    assert rel_err(z.grad.cpu().numpy(), gref) < TOL_F32


def test_autograd_batch_sums_instances():
    insts = cnfgen.batch_ksat(3, 4, n_lo=100, n_hi=400, k_hi=3)
    prob, st, cnfs = make(insts, 32)
    hp = ts.hparams(seed=1, norm=1)
    z = (torch.randn(prob.info["n_vars"], 32, device="cuda") + 0.3).requires_grad_(True)
    loss, S = SatObjective.apply(z, st, hp, 0)
    loss.backward()
    zc = z.detach().cpu().numpy()
    nu = st.view("nu").cpu().numpy()
    total = 0.0
    for j, cnf in enumerate(cnfs):
        a, b = prob.var_offsets[j], prob.var_offsets[j + 1]
        X = oracle.binarize_f32(zc[a:b], nu[a:b], 0)
        _, L, G, _ = oracle.objective(cnf, X=X, tau=1.0)
        total += L
        gj = oracle.normalize_backward(zc[a:b].astype(np.float64), nu[a:b].astype(np.float64), G, 1)
        assert rel_err(z.grad[a:b].cpu().numpy(), gj) < TOL_F32
    assert abs(loss.item() - total) < TOL_F32 * abs(total)


def test_relaxed_autograd_directional_fd():
    inst = cnfgen.structured_mixed(6000, 24000, 9, communities=12)
    prob, st, _ = make([inst], 32, layer=ts.LAYER_RELAXED)
    hp = ts.hparams(seed=2, norm=1, layer=ts.LAYER_RELAXED)
    g = torch.Generator(device="cuda").manual_seed(5)
    z = (torch.randn(6000, 32, device="cuda", generator=g) + 0.2).requires_grad_(True)
    loss, S = SatObjective.apply(z, st, hp, 0)
    loss.backward()
    rows = torch.randperm(6000, generator=torch.Generator().manual_seed(3))[:5000].cuda()
    d = torch.zeros_like(z)
    d[rows] = torch.sign(z.grad[rows])
    h = 1e-2
    with torch.no_grad():
        Lp, Sp = SatObjective.apply(z + h * d, st, hp, 0)
        Lm, _ = SatObjective.apply(z - h * d, st, hp, 0)
    fd = (Lp.item() - Lm.item()) / (2 * h)
    an = float((z.grad * d).sum().item())
    noise = 2 * 4e-6 * float(Sp.abs().sum().item()) / (2 * h)
    assert abs(fd - an) <= 1e-3 * abs(an) + noise, (fd, an, noise)


def test_torch_adamw_step_matches_fused_step():
    """One torch.optim.AdamW step driven by SatObjective equals the library's
    fused step from the same state (t = 0, lr 0.1, wd 0.01)."""
    inst = cnfgen.planted_ksat(1200, 5112, 3, 41)
    prob, st, cnfs = make([inst], 128)
    hp = ts.hparams(seed=6, norm=1, tau=1.0)
    ts.tsat_init(st.h, hp)
    s0 = snapshot(st)
    _, st2, _ = make([inst], 128)
    z = torch.tensor(s0["z"], device="cuda").requires_grad_(True)
    opt = torch.optim.AdamW([z], lr=0.1, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.01)
    loss, _ = SatObjective.apply(z, st2, hp, 0)
    opt.zero_grad()
    loss.backward()
    opt.step()
    ts.tsat_step(st.h, hp, 1, stop_on_sat=False)
    s1 = snapshot(st)
    st_opt = opt.state[z]
    assert_adamw_z(s1["z"], z.detach().cpu().numpy().astype(np.float64), s1["m"],
                   st_opt["exp_avg"].cpu().numpy().astype(np.float64), s1["v"],
                   st_opt["exp_avg_sq"].cpu().numpy().astype(np.float64), 0, hp)
