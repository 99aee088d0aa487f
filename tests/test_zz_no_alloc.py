"""The allocation-free entry point, for callers that cannot allocate device
memory (pooled or arena-owned device memory, no allocation during graph
construction, allocate-at-start-up hosts).  hf_increment_norms_noalloc
computes the Newton increment norms from caller-owned device vectors with a
fixed scratch array instead of an allocation; its result must match the
relative increments hf_newton_step reports (computed with the handle's
allocated scratch), on two calls in a row.  This file is collected last."""
import ctypes

import numpy as np
import pytest

from hf_inputs import kgd_2d
from _setup import gpu_for

pytestmark = pytest.mark.gpu


def test_noalloc_norms_match_newton_step_on_two_calls():
    torch = pytest.importorskip("torch")
    import paper_1911_10275_gb300 as pkg
    lib = pkg.load()
    wl = kgd_2d(n=8, length=16.0, steps=1, seed_cells=2)
    g = gpu_for(wl)
    g.hf_set_state(*wl.seed())
    err = ctypes.create_string_buffer(256)
    for call in range(2):
        U0, P0 = g.hf_get_state()[:2]
        rep = g.hf_newton_step()
        U1, P1 = g.hf_get_state()[:2]
        x1 = torch.tensor(np.concatenate([U1, P1]), dtype=torch.float64, device="cuda")
        x0 = torch.tensor(np.concatenate([U0, P0]), dtype=torch.float64, device="cuda")
        dx = x1 - x0
        out = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        st = lib.hf_increment_norms_noalloc(dx.data_ptr(), x1.data_ptr(), g.n_u, g.n_p, out.data_ptr(),
                                            stream, err, 256)
        assert st == 0, err.value
        torch.cuda.synchronize()
        s = out.cpu().numpy()
        du = np.sqrt(s[0]) / np.sqrt(s[1])
        dp = np.sqrt(s[2]) / np.sqrt(s[3])
        assert du == pytest.approx(rep["du_rel"], rel=1e-12, abs=1e-300)
        assert dp == pytest.approx(rep["dp_rel"], rel=1e-12, abs=1e-300)
    # sizes beyond the fixed scratch are refused before any device work
    st = lib.hf_increment_norms_noalloc(dx.data_ptr(), x1.data_ptr(), 1 << 26, 1, out.data_ptr(), None, err, 256)
    assert st == -1 and b"exceed" in err.value
    g.close()


def test_noalloc_norms_multi_block_and_empty():
    """Vectors spanning 3.5 scratch blocks of 16,384 unknowns with the
    displacement/pressure split inside the third block: the last-block sum
    over the block partials matches torch's sums, on two calls in a row (the
    ticket is cleared per call); an empty call writes zeros."""
    torch = pytest.importorskip("torch")
    import paper_1911_10275_gb300 as pkg
    lib = pkg.load()
    chunk = 16384
    n_u = 2 * chunk + 5000
    n = int(3.5 * chunk)
    n_p = n - n_u
    gen = torch.Generator(device="cuda").manual_seed(11)
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        dx = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
        x = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen) * 3.0
        out = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
        st = lib.hf_increment_norms_noalloc(dx.data_ptr(), x.data_ptr(), n_u, n_p, out.data_ptr(), stream, err, 256)
        assert st == 0, err.value
        torch.cuda.synchronize()
        want = torch.stack([(dx[:n_u] ** 2).sum(), (x[:n_u] ** 2).sum(), (dx[n_u:] ** 2).sum(),
                            (x[n_u:] ** 2).sum()]).cpu().numpy()
        assert np.allclose(out.cpu().numpy(), want, rtol=1e-12, atol=0)
    out = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    st = lib.hf_increment_norms_noalloc(dx.data_ptr(), x.data_ptr(), 0, 0, out.data_ptr(), stream, err, 256)
    assert st == 0, err.value
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), np.zeros(4))
