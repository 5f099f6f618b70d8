"""Config 4: beta = 1/2, N = 256, k = 16, 8192 bits.  lambda_1 and
d lambda_1 / d beta through torch.autograd (paper_1810_01478_gb300.lambda1),
against the oracle's values stored in tests/golden/c2.json (its analytic
gradient and its central finite difference at beta +- 1e-30 agree to ~1e-56)."""
import json
import os

import pytest

mpm = pytest.importorskip("mpmath")

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_autograd_gradient_config4():
    import torch
    import paper_1810_01478_gb300 as hk
    gd = json.load(open(os.path.join(HERE, "golden", "c2.json")))
    beta = torch.tensor(0.5, dtype=torch.float64, requires_grad=True)
    lam = hk.lambda1(beta, 256, 16, 8192)
    lam.backward()
    with mpm.workprec(200):
        want_l = mpm.mpf(gd["lambdas"][0])
        want_g = mpm.mpf(gd["grad"])
        assert abs(mpm.mpf(float(lam.detach())) - want_l) / want_l < 1e-15
        assert abs(mpm.mpf(float(beta.grad)) - want_g) / abs(want_g) < 1e-15
        # the finite difference of the oracle pipeline agrees as well
        assert abs(mpm.mpf(float(beta.grad)) - mpm.mpf(gd["grad_fd"])) / abs(want_g) < 1e-15


def test_autograd_rejects_irrational_beta():
    import torch
    import paper_1810_01478_gb300 as hk
    with pytest.raises(ValueError):
        hk.lambda1(torch.tensor(0.3183098861837907, dtype=torch.float64), 48, 8, 4096)
