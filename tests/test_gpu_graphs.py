"""Single-lattice steps inside CUDA graphs: lbm_run captured on a stream and replayed gives
the states of direct launches, for every precision form."""
import pytest
import torch

from paper_1703_04594_gb300 import lbm
from tests.gpu_util import device_init, require_gpu, rt_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP64_FIXED, lbm.FP32_SHIFTED])
def test_steps_replay_in_a_cuda_graph(precision):
    """lbm_run captured in a CUDA graph on a side stream and replayed gives the same states
    as direct launches (an even step count keeps the ping-pong parity)."""
    p = lbm.Params(64, 128, precision=precision)
    fields = rt_fields(p, seed=14)
    fa = device_init(p, fields)
    start = fa.clone()
    fb = lbm.empty_state(p)
    want = lbm.run(p, fa.clone(), lbm.empty_state(p), 8)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        lbm.run(p, fa, fb, 2, stream=s)                      # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    fa.copy_(start)
    with torch.cuda.graph(g):
        lbm.run(p, fa, fb, 4)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(fa[:, :, : p.ly], want[:, :, : p.ly])
