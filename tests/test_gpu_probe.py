"""The FMA-rate probe that the bench quotes ALU-bound kernels against: its
chains compute what they claim (x <- x a + b, iterated), so the flop count the
bench divides by is real work."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def probe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_03487_gb300 import measure
    return measure


@pytest.mark.parametrize("prec", [0, 1])
def test_fma_chains(probe, prec):
    blocks, iters = 3, 200
    dt = torch.float64 if prec == 0 else torch.float32
    sink = torch.empty(blocks * 256, dtype=dt, device="cuda")
    probe.fma_probe(sink, prec, iters, blocks)
    got = sink.cpu().numpy()
    a, b = (0.999999, 1e-6) if prec == 0 else (np.float32(0.9999), np.float32(1e-4))
    npdt = np.float64 if prec == 0 else np.float32
    tid = np.arange(blocks * 256)
    x = np.stack([(tid % 97).astype(npdt) * npdt(1e-3) + npdt(k) for k in range(8)])
    for _ in range(iters):
        x = (x * npdt(a) + npdt(b)).astype(npdt)
    expect = x.sum(axis=0)
    tol = 1e-12 if prec == 0 else 1e-5
    assert np.max(np.abs(got - expect) / np.abs(expect)) < tol
