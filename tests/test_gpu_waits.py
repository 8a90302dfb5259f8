"""Bounded inter-CTA waits (decoupled look-back of the sorts): with a poll
budget of one, a CTA whose predecessor has not published yet gives up; the
device status then reports GS_ERR_TIMEOUT, the render kernels of the chain
skip their work, nothing faults, and the same workspace renders correctly
again with the default budget."""
import numpy as np
import pytest
import torch

from paper_2506_00225_gb300 import _native as N
from paper_2506_00225_gb300 import raster, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00225_gb300 import build
    build.build()


def test_lookback_wait_runs_out_and_is_reported():
    w = scenes.workload("room300k")
    g = raster.Gaussians.from_scene(w["scene"])
    cam = w["cams"][0]
    with torch.no_grad():
        ref = [t.clone() for t in raster.Rasterizer().forward(g, cam, check=True)]
    rast = raster.Rasterizer(spin_limit=1)
    timed_out = False
    for _ in range(3):  # a predecessor may, rarely, always be ready in time
        try:
            with torch.no_grad():
                out = rast.forward(g, cam, check=True)
        except N.GsError as e:
            assert e.code == N.GS_ERR_TIMEOUT, e
            timed_out = True
            break
        for a, b in zip(out, ref):  # no wait ran out: the result is exact
            np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    assert timed_out
    torch.cuda.synchronize()  # the context is healthy
    rast.spin_limit = 0
    with torch.no_grad():
        out = rast.forward(g, cam, check=True)
    for a, b in zip(out, ref):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
