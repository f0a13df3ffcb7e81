"""The usage example in README.md runs as written on the GPU."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu

README = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "README.md")


def test_readme_example_runs():
    with open(README) as fh:
        blocks = re.findall(r"```python\n(.*?)```", fh.read(), flags=re.S)
    assert len(blocks) == 1
    scope = {}
    exec(compile(blocks[0], "README.md", "exec"), scope)
    assert scope["ll"] < 0 and len(scope["grad"]) == 6 and scope["pi"].shape[0] == 8
    assert abs(scope["ll"] - scope["ll64"]) <= 1e-6 * abs(scope["ll64"])
    assert abs(scope["ll_t"] - scope["ll"]) <= 1e-9 * abs(scope["ll"])
    assert len(scope["g2"]) == 9 and scope["ll2"] < 0
