"""The device modulo behind every row index (Sec. 2.2: one wide hash, then its
remainder modulo each block's Bloom size), a Barrett reduction with the
per-block constant floor(2^64 / w), compared with the integer remainder x % w
at edge widths and edge values, through the C ABI test hook."""
import numpy as np
import pytest

from paper_1905_09624_gb300 import cobs

pytestmark = pytest.mark.gpu

WIDTHS = sorted({1, 2, 3, 5, 7, 13, 255, 256, 257, 13935, 369_121, 910_307, 2_097_152}
                | {(1 << k) + d for k in (4, 8, 13, 16, 20, 24, 28, 31) for d in (-1, 0, 1)}
                | {1 << 31, (1 << 31) + 1, (1 << 32) - 3, (1 << 32) - 2, (1 << 32) - 1})


def _edge_values(w):
    top = (1 << 64) - 1
    v = {0, 1, w - 1, w, w + 1, 2 * w - 1, 2 * w, top, top - 1, top - w, top - w + 1, 1 << 63, (1 << 63) - 1,
         (1 << 32) - 1, 1 << 32}
    q = top // w
    v |= {q * w, q * w - 1, (q - 1) * w, (q - 1) * w + w - 1}
    return [x for x in v if 0 <= x <= top]


@pytest.mark.parametrize("w", WIDTHS)
def test_barrett_mod_equals_remainder(w):
    import torch
    torch.cuda.set_device(0)
    rng = np.random.default_rng(w)
    x = np.concatenate([rng.integers(0, np.iinfo(np.uint64).max, size=1_000_000, dtype=np.uint64, endpoint=True),
                        np.array(_edge_values(w), dtype=np.uint64)])
    d_x = torch.from_numpy(x.view(np.int64)).cuda()
    d_out = torch.full((len(x),), -1, dtype=torch.int32, device="cuda")
    cobs.debug_barrett_mod(d_x.data_ptr(), len(x), w, d_out.data_ptr())
    torch.cuda.synchronize()
    got = d_out.cpu().numpy().view(np.uint32).astype(np.uint64)
    want = x % np.uint64(w)
    bad = np.nonzero(got != want)[0]
    assert len(bad) == 0, (w, [(int(x[i]), int(got[i]), int(want[i])) for i in bad[:5]])


def test_barrett_mod_rejects_bad_widths():
    import torch
    L = cobs.lib()
    buf = torch.zeros(4, dtype=torch.int64, device="cuda")
    for w in (0, 1 << 32):
        assert L.cobs_debug_barrett_mod(buf.data_ptr(), 4, w, buf.data_ptr(), None) == cobs.COBS_ERR_ARG
