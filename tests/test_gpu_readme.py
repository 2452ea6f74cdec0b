"""The README's usage example runs as written (GPU)."""

import os
import re

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example_runs():
    assert torch.cuda.is_available()
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert blocks, "README has no python example"
    scope = {}
    exec(compile(blocks[0], "README.md", "exec"), scope)
    rho = scope["rho"]
    assert rho.shape == (3, 2, 2)
    for r in rho:
        assert abs(np.trace(r) - 1.0) < 1e-5
        assert np.abs(r - r.conj().T).max() < 1e-5
