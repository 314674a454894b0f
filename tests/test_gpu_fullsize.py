"""Full-size parity on the 1024 x 1024 workload (21 x 21 random-walk motion
blur, 1004 x 1004 valid crop with 40% of its pixels missing, BSNR 40 dB,
lambda 2e-6, mu 1e-3) in the launch configuration the benchmark times:
relative L2 <= 1e-5 after one iteration, and <= 1e-3 with |dPSNR| <= 0.01 dB
after the full 500 iterations, against the FP64 oracle."""
import numpy as np
import pytest

from paper_1602_01410_gb300 import inputs

from gpu_helpers import gpu_solve, oracle_solve, psnr, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def c2():
    return inputs.config_c2()


def test_c2_one_iteration(c2):
    xg, _, _ = gpu_solve(c2, iters=1)
    xo, _ = oracle_solve(c2, iters=1)
    assert rel_l2(xg, xo) <= 1e-5


def test_c2_full_run(c2):
    xg, _, _ = gpu_solve(c2)
    xo, _ = oracle_solve(c2)
    err = rel_l2(xg, xo)
    xt = c2.x_true[0]
    dpsnr = psnr(xg[0], xt) - psnr(xo[0], xt)
    print(f"c2 full run: rel L2 {err:.3e}, dPSNR {dpsnr:+.4f} dB")
    assert err <= 1e-3
    assert abs(dpsnr) <= 0.01
