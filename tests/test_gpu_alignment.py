"""Parameter arrays that do not start on a 16-byte boundary.

The projection kernels move each block's SH coefficients (and the backward
projection its SH gradients) with 16-byte vector accesses when the arrays
allow it, and element by element otherwise; both forms must give the same
renders and gradients.  The scene's size is no multiple of the 128-Gaussian
block, so the last block's tail is exercised too.
"""
import numpy as np
import pytest
import torch

import synthetic
from _helpers import KEYS, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_08174_gb300 import build
    build.build()
    return torch.device("cuda", 0)


def _offset_copy(t: torch.Tensor) -> torch.Tensor:
    """A contiguous copy of t whose data starts 4 bytes past a 16-byte boundary."""
    buf = torch.empty(t.numel() + 1, dtype=t.dtype, device=t.device)
    v = buf[1:].view(t.shape)
    v.copy_(t)
    assert v.data_ptr() % 16 == 4 and v.is_contiguous()
    return v


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_misaligned_sh_gives_the_same_render_and_gradients(dev, deg):
    from paper_2501_08174_gb300 import Rasterizer
    sc = synthetic.small_scene(801 + deg, 1000, 70, 45, degree=deg, n_views=2)
    g = to_device(sc["gaussians"], dev)
    assert g["sh"].data_ptr() % 16 == 0
    g_off = dict(g, sh=_offset_copy(g["sh"]))
    r = Rasterizer(dev)
    outs, grads = [], []
    rng = np.random.default_rng(deg)
    P = sum(c["width"] * c["height"] for c in sc["cameras"])
    d = {"rgb": torch.tensor(rng.normal(size=(P, 3)), dtype=torch.float32, device=dev),
         "alpha": torch.tensor(rng.normal(size=P), dtype=torch.float32, device=dev)}
    for gg, aligned in ((g, True), (g_off, False)):
        score = torch.zeros(g["opacity"].shape[0], device=dev)
        out, st = r.render(gg, sc["cameras"], score=score)
        gr = {k: torch.zeros_like(gg[k]) for k in KEYS}
        if not aligned:
            gr["sh"] = _offset_copy(gr["sh"])
        r.render_backward(st, gg, d, grads=gr)
        st.release()
        torch.cuda.synchronize()
        outs.append(({k: v.cpu() for k, v in out.items()}, score.cpu()))
        grads.append({k: v.cpu() for k, v in gr.items()})
    r.close()
    (a, sa), (b, sb) = outs
    for k in a:
        assert torch.equal(a[k], b[k]), k
    assert torch.equal(sa, sb)
    for k in KEYS:  # float atomics in the backward rasterizer: equal up to their summation order
        ref = grads[0][k]
        assert torch.allclose(grads[1][k], ref, rtol=1e-5, atol=1e-6 * float(ref.abs().max())), k
    assert float(grads[0]["sh"].abs().max()) > 0
