"""The remaining entry points on the GPU: the copy-19 / update-19 bandwidth
micro-benchmarks (exact results, padding untouched), the FP64 FMA probe, and
the handle queries (fluid count, device bytes, step count, synchronize)."""
import numpy as np
import pytest

from paper_1711_11468_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("elem", [2, 4, 8])
def test_copy19_and_update19_exact(lbm, elem):
    import torch
    dtype = {2: torch.int16, 4: torch.int32, 8: torch.int64}[elem]
    n, stride = 100_003, 100_003 + 61   # ragged length, padded arrays
    g = torch.Generator().manual_seed(elem)
    src = torch.randint(-1000, 1000, (19 * stride,), generator=g, dtype=dtype).cuda()
    dst = torch.full((19 * stride,), 7, dtype=dtype, device="cuda")
    s = torch.cuda.current_stream()
    lbm.lbm_bench_copy19(src.data_ptr(), dst.data_ptr(), n, stride, elem, s)
    before = dst.clone()
    lbm.lbm_bench_update19(dst.data_ptr(), n, stride, elem, s)
    torch.cuda.synchronize()
    a, b, c = src.view(19, stride).cpu(), before.view(19, stride).cpu(), dst.view(19, stride).cpu()
    assert torch.equal(b[:, :n], a[:, :n])
    assert torch.all(b[:, n:] == 7)            # the padding is not written
    assert torch.equal(c[:, :n], a[:, :n] + 1)
    assert torch.all(c[:, n:] == 7)


def test_fma64_probe(lbm):
    import torch
    blocks = lbm.lbm_bench_fma64_wave()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert blocks >= sms and blocks % sms == 0
    out = torch.zeros(blocks * 256, dtype=torch.float64, device="cuda")
    lbm.lbm_bench_fma64(out.data_ptr(), blocks, 3, torch.cuda.current_stream())
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    # 16 chains a <- a * b + c from a = 1 + 1e-3 (thread + k), three times
    t = np.arange(blocks * 256) % 256
    want = np.zeros(blocks * 256)
    b, c = 0.9999999, 1e-7
    for k in range(16):
        a = 1.0 + 1e-3 * (t + k)
        for _ in range(3):
            a = a * b + c
        want += a
    assert np.allclose(got, want, rtol=1e-14, atol=0)


def test_handle_queries(lbm, orc):
    import torch
    dims = (24, 18, 20)
    fl = inputs.channel_flags(*dims)
    for addr, fluid in ((lbm.LBM_DIRECT, fl), (lbm.LBM_INDIRECT, np.where(fl == 1, 2, 0).astype(np.uint8))):
        h = lbm.lbm_create_lattice(lbm.make_desc(dims, lbm.LBM_F64, addr, lbm.LBM_AA_INPLACE, (1, 0, 1)),
                                   torch.cuda.current_stream())
        try:
            lbm.lbm_set_geometry(h, 0, fluid)
            nf = int((fluid == 0).sum())
            assert lbm.lbm_fluid_count(h, 0) == nf
            # the PDFs alone take 19 arrays of at least N (direct) or N_f (list) doubles
            assert lbm.lbm_memory_bytes(h) >= 19 * 8 * (np.prod(dims) if addr == lbm.LBM_DIRECT else nf)
            lbm.lbm_set_params(h, 0, 1.1, 0.25, (1e-6, 0.0, 0.0))
            lbm.lbm_init_equilibrium(h, 0)
            assert lbm.lbm_steps_done(h) == 0
            lbm.lbm_step(h, 5)
            lbm.lbm_synchronize(h)
            assert lbm.lbm_steps_done(h) == 5
            f = lbm.lbm_read_pdfs(h, 0)
            lbm.lbm_write_pdfs(h, 0, f)
            assert lbm.lbm_steps_done(h) == 0
        finally:
            lbm.lbm_destroy(h)
