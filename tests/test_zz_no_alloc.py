"""residual_loss_static: the loss for callers that cannot allocate device
memory (no workspace argument; scratch in a fixed array inside the library).

Checked through the C ABI against residual_loss with a workspace, on two
calls in a row, with the tolerances of the residual-loss parity test.  This
file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

GPU = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2606_08469_gb300 import build
    build.build()
    from paper_2606_08469_gb300 import _lib
    return _lib.load()


def test_static_loss_rejects_batches_beyond_its_scratch(lib):
    from paper_2606_08469_gb300 import _lib as L
    rc = lib.residual_loss_static(None, None, None, None, 2_796_203, C.c_float(0.01), 1, None,
                                  None, None, None, None)
    assert rc == L.OCTA_ERANGE
    assert b"fixed scratch limit" in lib.octa_last_error()


@GPU
def test_static_loss_matches_workspace_loss_twice(lib):
    from paper_2606_08469_gb300 import _lib as L
    from paper_2606_08469_gb300 import api as A
    dev = "cuda"
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: C.c_void_p(t.data_ptr())
    for call, n in enumerate((262_144, 70_001)):        # two calls in a row
        g = np.random.default_rng(100 + call)
        Lp, Ls = (torch.from_numpy(g.uniform(0.2, 3.0, size=(n, 3)).astype(np.float32)).to(dev)
                  for _ in range(2))
        E = torch.from_numpy((g.random((n, 3)) * (g.random((n, 1)) < 0.05)).astype(np.float32)).to(dev)
        w = torch.from_numpy(g.random((n, 3)).astype(np.float32)).to(dev)
        scaler = A.make_scaler(2.0 ** 15, 2000)
        ws = A.workspace(L.OCTA_OP_LOSS, n)
        ref = [torch.zeros(1, dtype=torch.float64, device=dev), torch.empty((n, 3), device=dev),
               torch.empty((n, 3), device=dev)]
        got = [torch.zeros(1, dtype=torch.float64, device=dev), torch.empty((n, 3), device=dev),
               torch.empty((n, 3), device=dev)]
        L.check(lib.residual_loss(p(Lp), p(Ls), p(E), p(w), n, C.c_float(1e-2), 1, p(scaler),
                                  p(ref[0]), p(ref[1]), p(ref[2]), p(ws), ws.numel(), stream),
                "residual_loss")
        L.check(lib.residual_loss_static(p(Lp), p(Ls), p(E), p(w), n, C.c_float(1e-2), 1,
                                         p(scaler), p(got[0]), p(got[1]), p(got[2]), stream),
                "residual_loss_static")
        torch.cuda.synchronize()
        assert abs(got[0].item() - ref[0].item()) <= 1e-6 * ref[0].item()
        torch.testing.assert_close(got[1], ref[1], rtol=2e-5, atol=0)
        torch.testing.assert_close(got[2], ref[2], rtol=2e-5, atol=0)
