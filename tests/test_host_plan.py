"""The host-side numbers of the CUDA path against the oracle, on the CPU
(no device work): the Legendre-zero schedule of App. A.5, the RKL stage
coefficients the kernels run (App. A; RKL2 of the a_s + b_s P_s family), the
level rule of Sec. 4.1, App. B's SOR omega and App. A.4's global s_opt.  The C++ and the oracle are
written separately; schedules and level counts must agree exactly, the
coefficients to a few ulps."""

import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def sg():
    import paper_2306_05332_gb300 as sg
    if not __import__("os").path.exists(sg.LIB_PATH):
        from paper_2306_05332_gb300 import build
        build.build()
    sg.lib()
    return sg


@pytest.mark.parametrize("N", [2, 3, 4, 6, 8, 12, 16, 20, 24, 32, 48, 64, 96, 128, 256, 512])
def test_schedule_matches_oracle(sg, N):
    count = N + 12
    assert sg.plan_schedule(N, count) == O.accelerated_schedule(N, count)


@pytest.mark.parametrize("order,s", [(1, 1), (1, 2), (1, 7), (1, 24), (1, 97), (2, 2), (2, 3), (2, 4),
                                     (2, 6), (2, 13), (2, 40)])
def test_stage_coefficients_match_oracle(sg, order, s):
    c = sg.plan_stage_coefficients(order, s)
    ref = O.rkl_coefficients(order, s)
    for name, r in (("mu", ref.mu), ("nu", ref.nu), ("mut", ref.mu_t), ("gt", ref.gamma_t)):
        np.testing.assert_allclose(c[name][1:], r[1:], rtol=4e-16, atol=1e-300, err_msg=name)
    assert abs(c["tau_max_over_dtpar"] - ref.tau_max_over_dtpar) <= 1e-15 * ref.tau_max_over_dtpar


@pytest.mark.parametrize("shape", [(256, 256, 256), (96, 96, 96), (32, 32, 32), (8, 4, 6), (12, 12, 12),
                                   (24, 32, 48), (40, 24, 72), (2, 2, 2), (9, 36, 13), (64, 128, 256)])
def test_level_rule_matches_oracle(sg, shape):
    assert sg.plan_levels(shape) == O.level_count(shape)


@pytest.mark.parametrize("shape,lo,hi", [((32, 32, 32), (0, 0, 0), (1, 1, 1)),
                                         ((16, 24, 40), (0.0, -0.5, 0.25), (1.3, 0.2, 1.35)),
                                         ((128, 128, 128), (-0.5,) * 3, (0.5,) * 3)])
def test_sor_omega_matches_oracle(sg, shape, lo, hi):
    om = sg.plan_sor_omega(shape, lo, hi)
    assert abs(om - O.sor_omega(shape, O.spacing(shape, lo, hi))) < 1e-14


@pytest.mark.parametrize("N", [2, 3, 4, 8, 16, 24, 32, 48, 64, 96, 100, 128, 200, 256, 512, 1024])
def test_global_s_opt_matches_oracle(sg, N):
    assert sg.plan_s_opt(N) == O.s_opt_global(N)


def test_planning_rejects_bad_arguments(sg):
    L = sg.lib()
    assert L.sg_plan_schedule(0, 3, None) == 1
    assert L.sg_plan_schedule(8, 3, None) == 1
    assert L.sg_plan_stage_coefficients(2, 1, None, None, None, None, None) == 1
    assert L.sg_plan_stage_coefficients(3, 5, None, None, None, None, None) == 1
    assert L.sg_plan_levels(0, 4, 4) == 0
    assert L.sg_plan_s_opt(1, None) == 1
    with pytest.raises(sg.SGError):
        sg.plan_sor_omega((8, 8, 8), (0, 0, 0), (1, 0, 1))
