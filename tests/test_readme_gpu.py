"""The README's usage example runs as written on the GPU and gives finite
losses and gradients."""
import math
import os

import pytest

pytestmark = pytest.mark.gpu


def test_readme_example_runs():
    from tests.gpu_util import gpu_lib
    gpu_lib()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "README.md")).read()
    code = text.split("```python")[1].split("```")[0]
    ns: dict = {}
    exec(compile(code, "README.md", "exec"), ns)
    import torch
    torch.cuda.synchronize()
    assert math.isfinite(float(ns["loss"].item()))
    assert ns["rho"].grad is not None and torch.isfinite(ns["rho"].grad).all()
    assert ns["ego"].grad is not None and torch.isfinite(ns["ego"].grad).all()
    plan = ns["plan"]
    assert torch.isfinite(plan.loss).all() and (plan.loss > 0).all()
    assert all(torch.isfinite(o["dego"]).all() for o in plan.outputs)
    det = ns["det"]
    torch.cuda.synchronize()
    # the deterministic plan agrees with the atomic one within the FP32 tolerances
    assert torch.allclose(det.loss, plan.loss, rtol=1e-5, atol=0)
