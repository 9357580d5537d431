"""fft_execute_host: host buffers in and out through the plan's staging
buffers, pipelined across calls.  Results must equal fft_execute on the same
input bit for bit (same kernels, same data)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_15437_gb300 import build
    build.build()
    import paper_2506_15437_gb300 as g
    return g


@pytest.mark.parametrize("nx,ny,batch", [(8192, 8192, 1), (1024, 512, 3), (1 << 16, 1, 4), (1000, 300, 2),
                                         (1 << 25, 1, 1), (10 ** 6, 1, 2)])
def test_host_round_trip_matches_device_path(g, nx, ny, batch):
    plan = g.Plan(nx, ny, batch)
    xs = [synth.uniform_complex((batch, ny, nx), seed=40 + k) for k in range(4)]
    hin = [torch.from_numpy(x).pin_memory() for x in xs]
    hout = [torch.empty_like(h).pin_memory() for h in hin]
    for k in range(4):  # four calls back to back: the staging buffers alternate
        plan.execute_host(hin[k], hout[k])
    torch.cuda.synchronize()
    assert plan.status() == 0
    for k in range(4):
        ref = plan.execute(hin[k].cuda()).cpu()
        assert torch.equal(torch.view_as_real(hout[k]), torch.view_as_real(ref)), k
    plan.close()


def test_host_rejects_device_and_aliased_buffers(g):
    plan = g.Plan(64, 64, 1)
    h = torch.zeros(64 * 64, dtype=torch.complex64).pin_memory()
    with pytest.raises(ValueError):
        plan.execute_host(h.cuda())
    from paper_2506_15437_gb300 import _native
    lib = _native.load()
    assert lib.fft_execute_host(plan._p, h.data_ptr(), h.data_ptr(), 0) == -2
    plan.close()


def test_host_calls_interleaved_with_device_calls(g):
    """Host calls (plan compute stream) and device calls (caller's stream)
    on one plan share its workspaces; interleaved, every result stays
    correct."""
    plan = g.Plan(8192, 8192, 1)
    xs = [synth.uniform_complex((8192, 8192), seed=60 + k) for k in range(4)]
    refs = []
    for k in range(4):
        hin = torch.from_numpy(xs[k]).pin_memory()
        if k % 2 == 0:
            hout = plan.execute_host(hin, torch.empty_like(hin).pin_memory())
        else:
            hout = plan.execute(hin.cuda()).cpu()
        refs.append(hout)
    torch.cuda.synchronize()
    for k in range(4):
        want = plan.execute(torch.from_numpy(xs[k]).cuda()).cpu()
        assert torch.equal(torch.view_as_real(refs[k]), torch.view_as_real(want)), k
    plan.close()


@pytest.mark.parametrize("nx,ny,batch", [(8192, 8192, 1), (1 << 24, 1, 1), (1003, 1003, 1), (1000, 1000, 1),
                                         (4096, 4096, 2)])
def test_execute_is_graph_capturable(g, nx, ny, batch):
    """fft_execute allocates and synchronises nothing, so a CUDA graph can
    capture it: the landed-pair rows with the streaming planar columns, the
    four-step path, the fused Bluestein path with its transposes and the
    mixed-radix path with its in-place column kernel.  A
    replay on new input gives the eager result bit for bit."""
    plan = g.Plan(nx, ny, batch)
    x0 = torch.from_numpy(synth.uniform_complex((batch, ny, nx), seed=81)).cuda()
    x1 = torch.from_numpy(synth.uniform_complex((batch, ny, nx), seed=82)).cuda()
    src = x0.clone()
    dst = torch.empty_like(src)
    plan.execute(src, out=dst)  # plan-level lazy state (tensor maps) settled before capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            plan.execute(src, out=dst)
    src.copy_(x1)
    graph.replay()
    torch.cuda.synchronize()
    want = plan.execute(x1)
    torch.cuda.synchronize()
    assert torch.equal(torch.view_as_real(dst), torch.view_as_real(want))
    assert plan.status() == 0
    plan.close()
