"""GPU parity of long 1D transforms (n = 2^14 .. 2^26, the four-step path)
against the FP64 oracle, through the C ABI via the ctypes binding.

Bar: relative L2 error per transform <= 2e-7 * log2(n).  Every size, up to
the bench's 2^24 x 4, 2^25 x 2 and 2^26 x 1 in both their three-pass and
two-pass forms, is compared whole with the oracle's recursive transform, and
the round trip inverse(forward(x)) = n x holds over the whole output.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import ORACLE_THREADS, rel_l2, tol_fp32, worst_rel_l2

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


def run(g, x, inverse=False, inplace=False):
    n = x.shape[-1]
    batch = x.size // n
    plan = g.get_plan(n, 1, batch, inverse, "fp32", "cuda")
    d = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = plan.execute(d, out=d if inplace else None)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return out.cpu().numpy(), plan


@pytest.mark.parametrize("L", list(range(14, 22)))
@pytest.mark.parametrize("inverse", [False, True])
def test_full_against_oracle(g, L, inverse):
    n = 1 << L
    x = synth.uniform_complex((2, n), seed=300 + L)
    got, plan = run(g, x, inverse)
    d = plan.describe()
    assert d["fourstep"]["n1"] * d["fourstep"]["n2"] == n
    ref = oracle.fft1d_batch(x, dir=1 if inverse else -1, threads=ORACLE_THREADS)
    err = worst_rel_l2(got, ref, n)
    assert err <= tol_fp32(n), (L, inverse, err)


def test_2p22_exp_mix(g):
    n = 1 << 22
    x, freqs = synth.exp_mix_1d(1, n, seed=2506)
    got, _ = run(g, x)
    ref = oracle.fft1d_batch(x, threads=ORACLE_THREADS)
    assert rel_l2(got, ref) <= tol_fp32(n)
    # the planted exponentials stand out at their own bins
    assert np.all(np.abs(got[0, freqs[0]]) > 0.5 * n)


def test_in_place(g):
    n = 1 << 16
    x = synth.uniform_complex((3, n), seed=77)
    got, _ = run(g, x, inplace=True)
    ref = oracle.fft1d_batch(x, threads=ORACLE_THREADS)
    assert worst_rel_l2(got, ref, n) <= tol_fp32(n)


def test_backward_is_the_opposite_sign_transform(g):
    n = 1 << 18
    gy = synth.uniform_complex((2, n), seed=91)
    plan = g.get_plan(n, 1, 2, False, "fp32", "cuda")
    d = torch.from_numpy(gy).cuda()
    got = plan.backward(d).cpu().numpy()
    ref = oracle.fft1d_batch(gy, dir=1, threads=ORACLE_THREADS)
    assert worst_rel_l2(got, ref, n) <= tol_fp32(n)


def test_fft1_autograd_matches_adjoint(g):
    n = 1 << 15
    x = torch.from_numpy(synth.uniform_complex((2, n), seed=5)).cuda().requires_grad_(True)
    w = torch.from_numpy(synth.mask((2, n), seed=6)).cuda()
    X = g.fft1(x)
    loss = (w * X.real ** 2 + w * X.imag ** 2).sum()
    loss.backward()
    # dL/dx = 2 F^H (w X), F^H = the opposite-sign unnormalised transform
    wX = w.cpu().numpy() * X.detach().cpu().numpy().astype(np.complex128)
    ref = 2.0 * oracle.fft1d_batch(wX, dir=1, threads=ORACLE_THREADS)
    assert worst_rel_l2(x.grad.cpu().numpy(), ref, n) <= 2 * tol_fp32(n)


def test_weighted_adjoint_unsupported(g):
    n = 1 << 14
    plan = g.get_plan(n, 1, 1, False, "fp32", "cuda")
    X = torch.zeros(n, dtype=torch.complex64, device="cuda")
    w = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(g.FFTError):
        plan.backward_weighted(X, w, 2.0)


_REF = {}


@pytest.mark.parametrize("L,batch,three", [(24, 4, "1"), (25, 2, "1"), (25, 2, "0"), (26, 1, "1"), (26, 1, "0")])
def test_large_full_against_oracle_and_roundtrip(g, monkeypatch, L, batch, three):
    """The bench's workloads: every output of every transform against the
    oracle's recursive transform of the same input, and inverse(forward(x))
    = n x over the whole output.  2^25 and 2^26 run three passes (a middle
    pass of 2 or 4 points between 4096-point columns and rows) unless
    GB300FFT_FS_THREE=0 keeps the two-pass split."""
    n = 1 << L
    x = synth.uniform_complex((batch, n), seed=2506)
    monkeypatch.setenv("GB300FFT_FS_THREE", three)
    fwd = g.Plan(n, 1, batch)
    inv = g.Plan(n, 1, batch, inverse=True)
    monkeypatch.delenv("GB300FFT_FS_THREE")
    fsd = fwd.describe()["fourstep"]
    assert fsd["m"] == (n >> 24 if L >= 25 and three == "1" else 1)
    d = torch.from_numpy(x).cuda()
    X = fwd.execute(d)
    back = inv.execute(X)
    torch.cuda.synchronize()
    assert fwd.status() == 0 and inv.status() == 0
    tol = tol_fp32(n)
    if L not in _REF:
        _REF[L] = oracle.fft1d_batch(x, threads=ORACLE_THREADS)
    err = worst_rel_l2(X.cpu().numpy(), _REF[L], n)
    print(f"2^{L} x {batch} (three-pass={three}): whole-output rel L2 {err:.3e} (bound {tol:.2e})")
    assert err <= tol
    rt = back.cpu().numpy()
    assert worst_rel_l2(rt, n * x.astype(np.complex128), n) <= 2 * tol
    fwd.close()
    inv.close()


@pytest.mark.parametrize("L", [25, 26])
def test_three_pass_matches_two_pass(g, monkeypatch, L):
    """The three-pass and two-pass forms of the same transform share no pass
    schedule (4096 x M x 4096 against 8192 x 4096 or 8192 x 8192): every
    output agrees within twice the FP32 bound, both directions."""
    n = 1 << L
    x = torch.from_numpy(synth.uniform_complex((1, n), seed=77 + L)).cuda()
    for inverse in (False, True):
        three = g.Plan(n, 1, 1, inverse=inverse)
        monkeypatch.setenv("GB300FFT_FS_THREE", "0")
        two = g.Plan(n, 1, 1, inverse=inverse)
        monkeypatch.delenv("GB300FFT_FS_THREE")
        assert three.describe()["fourstep"]["m"] == n >> 24 and two.describe()["fourstep"]["m"] == 1
        a = three.execute(x)
        b = two.execute(x)
        c = x.clone()
        three.execute(c, out=c)  # in place: the first pass reads the input whole, the last writes it
        torch.cuda.synchronize()
        err = (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()
        assert err <= 2 * tol_fp32(n), (L, inverse, err)
        assert torch.equal(torch.view_as_real(c), torch.view_as_real(a))
        three.close()
        two.close()
