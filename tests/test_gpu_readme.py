"""The usage example of the README runs as written (order-20 scene forward,
autograd through the reverse mode, a batched launch)."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example_runs():
    import torch
    with open(os.path.join(ROOT, "README.md")) as f:
        block = re.search(r"```python\n(.*?)```", f.read(), re.S).group(1)
    scope = {}
    exec(compile(block, "README.md", "exec"), scope)
    torch.cuda.synchronize()
    x, params, beta, y, ys = (scope[k] for k in ("x", "params", "beta", "y", "ys"))
    assert y.shape == (1, x.numel())
    for g in (x.grad, params.grad, beta.grad):
        assert g is not None and bool(torch.isfinite(g).all())
    assert len(ys) == 4 and all(bool(torch.isfinite(v).all()) for v in ys)
