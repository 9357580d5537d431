"""Plans of every kind created from several host threads at once, in a
fresh process (the kernel registries are filled on first use): every plan
is valid and gives the same bits as one created alone afterwards."""
import os
import subprocess
import sys
import textwrap

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import sys, threading
    sys.path.insert(0, {root!r})
    import torch, synth
    import paper_2506_15437_gb300 as g
    torch.cuda.init()
    shapes = [(8192, 8192, 1, "fp32"), (4096, 1, 64, "fp32"), (1 << 16, 1, 2, "fp32"), (1000, 300, 1, "fp32"),
              (4095, 1, 4, "fp32"), (1024, 1024, 1, "split_tc"), (20000, 1, 1, "fp32"), (256, 256, 3, "fp32")]
    plans = [None] * len(shapes)
    errors = []
    def make(k):
        try:
            torch.cuda.set_device(0)
            nx, ny, b, prec = shapes[k]
            plans[k] = g.Plan(nx, ny, b, precision=prec)
        except Exception as e:  # reported below
            errors.append((k, repr(e)))
    ts = [threading.Thread(target=make, args=(k,)) for k in range(len(shapes))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    for k, (nx, ny, b, prec) in enumerate(shapes):
        x = torch.from_numpy(synth.uniform_complex((b, ny, nx), seed=k)).cuda()
        a = plans[k].execute(x)
        alone = g.Plan(nx, ny, b, precision=prec)
        ref = alone.execute(x)
        torch.cuda.synchronize()
        assert plans[k].status() == 0, k
        assert torch.equal(torch.view_as_real(a), torch.view_as_real(ref)), k
        plans[k].close()
        alone.close()
    print("threads ok")
""")


def test_plans_created_concurrently():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_15437_gb300 import build
    build.build()
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "threads ok" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
