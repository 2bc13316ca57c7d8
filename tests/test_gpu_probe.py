"""The integer-mix probe (a measurement aid for the pair check's roofline):
its output must equal the same word operation carried out in numpy, so the
timed launches do all the work they are credited with."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def msm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_0904_3151_gb300 import build as b
    b.build()
    import paper_0904_3151_gb300 as m
    m.lib()
    return m


def _probe_numpy(blocks, iters, seed):
    e = np.arange(blocks * 256 * 8, dtype=np.uint64)
    chain = (e % 8).astype(np.uint32)
    a = ((e * np.uint64(0x9E3779B1) + np.uint64(seed)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    b = (((e * np.uint64(0x85EBCA6B)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
         ^ np.uint32(seed))
    g = np.where(chain & 1, np.uint32(0x80008000), np.uint32(0x8000)).astype(np.uint32)
    bad = np.zeros_like(a)
    with np.errstate(over="ignore"):
        for _ in range(iters):
            t = (a ^ b) + np.uint32(0x7FFF7FFF)
            bad |= g & ~t
            a = t
    return bad ^ a


@pytest.mark.parametrize("blocks,iters,seed", [(1, 0, 0), (3, 1, 7), (2, 517, 0xDEADBEEF)])
def test_int_mix_probe_matches_numpy(msm, blocks, iters, seed):
    import torch
    out = torch.full((blocks * 256 * 8,), -1, dtype=torch.int32, device="cuda")
    from paper_0904_3151_gb300 import probe
    probe.int_mix_probe(out, blocks, iters, seed)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, _probe_numpy(blocks, iters, seed))


def test_int_mix_probe_rejects_bad_arguments(msm):
    import ctypes
    from paper_0904_3151_gb300 import probe
    assert probe.load().msm_int_mix_probe(None, 1, 1, ctypes.c_uint32(0), None) == -1
