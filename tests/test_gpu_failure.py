"""Failure detection on the GPU without a GPU fault.

The persistent tensor-core kernel bounds every wait on its pipeline barriers.
Here a plan's wait limit is cut to 1 microsecond, far below the time one pass
of a P6 element needs to reach its accumulator, so the epilogue's first wait
must give up: the kernel then stops, drains what it issued, frees its tensor
memory and returns, and fe_sync_status reports FE_ERR_TIMEOUT.  The plan is
then used again with the default limit and must give results bitwise equal
to a clean run.  A coefficient far beyond FP16's range in the FP16 action is
reported as an overflow instead of producing infinities.
"""
import numpy as np
import pytest
import torch

from paper_2410_12614_gb300 import _lib, inputs

from gpu_util import cuda, make_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["bf16", "e4m3"])
def test_wait_limit_gives_up_and_plan_recovers(prec):
    plan, _, kap = make_case("tetrahedron", 4, 6, 0.15, 140, 141, precisions=(prec,))
    kd = cuda(kap)
    clean = plan.element_matrices(kd, prec=prec)
    plan.sync()
    clean = {f: t.clone() for f, t in clean.items()}
    plan.set_wait_limit(1000)   # 1 us per wait
    plan.element_matrices(kd, prec=prec)
    with pytest.raises(_lib.FeError) as e:
        plan.sync()
    assert e.value.status == -7, e.value
    plan.sync()                  # the status word was cleared
    plan.set_wait_limit(0)       # back to the default
    again = plan.element_matrices(kd, prec=prec)
    plan.sync()
    for f in clean:
        assert torch.equal(again[f], clean[f]), f
    # the assembled path recovers too
    v1 = plan.assemble(kd, prec=prec)
    plan.sync()
    v2 = plan.assemble(kd, prec=prec)
    plan.sync()
    for f in v1:
        assert torch.equal(v1[f], v2[f])


def test_fp16_action_overflow_is_reported():
    plan, _, kap = make_case("tetrahedron", 2, 2, 0.15, 150, 151, precisions=("bf16",))
    w = cuda(inputs.gaussian_vector(plan.n_dofs, 152).astype(np.float64))
    kap = kap.copy()
    kap[3, :] = 1.0e12           # every r_s of cell 3 is ~1e12 times its a-priori scale
    plan.action(cuda(kap), w, prec="fp16")
    with pytest.raises(_lib.FeError) as e:
        plan.sync()
    assert e.value.status == -4 and "overflow" in str(e.value)
    plan.sync()
    # BF16 has FP32's range: the same input is fine there
    plan.action(cuda(kap), w, prec="bf16")
    plan.sync()
