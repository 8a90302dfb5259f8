"""The streamed, graph-captured mapping step (pipeline.MappingStream)
returns, for every frame, the loss and gradients of the eager
render_l1 + backward on the same frame."""
import pytest
import torch

from paper_2506_00225_gb300 import raster, scenes
from gradtol import WIDE, grad_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00225_gb300 import build
    build.build()


def test_stream_matches_eager_steps():
    from paper_2506_00225_gb300 import pipeline
    sc = scenes.scene_plain(0, n=6000, m=40, k=3)
    cam = scenes.look_camera((0.0, 0.0, 1.5), 10.0, 96, 72, 60.0, pitch_deg=-5.0)
    g = raster.Gaussians.from_scene(sc)
    frames = []
    for seed in (11, 12, 13, 14, 15):
        tg = raster.Gaussians.from_scene(scenes.perturbed_copy(sc, seed))
        with torch.no_grad():
            t_rgb, t_depth, _, t_sem = raster.Rasterizer().forward(tg, cam)
        frames.append(tuple(t.clone() for t in (t_rgb, t_depth, t_sem)))
    # eager reference, one fresh step per frame
    ref = []
    rast_e = raster.Rasterizer()
    for tr, td, ts in frames:
        params = [t.clone().requires_grad_(True) for t in (g.means, g.scales, g.quats, g.opacity, g.rgb, g.sem_w)]
        loss = raster.render_l1(rast_e, g, cam, tr, td, ts, *params)
        loss.backward()
        ref.append((float(loss.detach()), [p.grad.clone() for p in params]))
    # streamed: pinned host frames, two slots, graphs
    rast = raster.Rasterizer()
    rast.forward(g, cam, check=True)
    params = [t.clone().requires_grad_(True) for t in (g.means, g.scales, g.quats, g.opacity, g.rgb, g.sem_w)]
    stream = pipeline.MappingStream(rast, g, cam, params, *frames[0])
    host = [tuple(t.cpu().pin_memory() for t in f) for f in frames]
    for i, (h_rgb, h_depth, h_sem) in enumerate(host):
        s = stream.step(h_rgb, h_depth, h_sem)
        torch.cuda.synchronize()
        lr, gr = ref[i]
        assert abs(stream.loss_host(s) - lr) <= 1e-6 * abs(lr), (i, stream.loss_host(s), lr)
        for a, b in zip(stream.grads[s], gr):
            a, b = a.cpu().numpy(), b.cpu().numpy()
            grad_close(a, b, 1e-4, floor=WIDE)
    # back-to-back steps without host synchronisation: the last loss is the
    # last frame's
    for h in host:
        s = stream.step(*h)
    torch.cuda.synchronize()
    assert abs(stream.loss_host(s) - ref[-1][0]) <= 1e-6 * abs(ref[-1][0])
