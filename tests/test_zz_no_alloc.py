"""The allocation-free entry point, fastged_batch_noalloc.

It exists for callers that cannot allocate device memory (an application that owns all
device memory through its own pool, a plugin with a fixed device budget): they pass device
inputs and outputs, and the library takes every scratch byte from a fixed device array it
carries. Its results must equal those of the ordinary entry point, fastged_batch_ex, on the
same batch - checked here on two calls in a row, since the scratch array keeps the previous
call's contents. This file is collected last so a failure here comes after every other test.
"""
import numpy as np
import pytest

from paper_2605_00830_gb300 import fastged as F
from paper_2605_00830_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _device_batch(w, torch):
    """The workload flattened into torch device tensors, and the struct describing them."""
    mm = F.marshal(w)
    dev = "cuda"
    keep = {}
    n = mm.n.astype(np.int32)
    m = mm.m.astype(np.int32)
    voff = np.zeros(len(n), np.int64)
    eoff = np.zeros(len(m), np.int64)
    if len(n):
        voff[1:] = np.cumsum(n[:-1])
        eoff[1:] = np.cumsum(m[:-1])
    keep["n"] = torch.from_numpy(n).to(dev)
    keep["m"] = torch.from_numpy(m).to(dev)
    keep["voff"] = torch.from_numpy(voff).to(dev)
    keep["eoff"] = torch.from_numpy(eoff).to(dev)
    keep["vl"] = torch.from_numpy(mm.vl.astype(np.int32)).to(dev)
    keep["ed"] = torch.from_numpy(mm.ed.astype(np.int32)).to(dev)
    keep["el"] = None if mm.el is None else torch.from_numpy(mm.el.astype(np.int32)).to(dev)
    keep["pairs"] = torch.from_numpy(mm.pairs.reshape(-1)).to(dev)
    keep["moff"] = torch.from_numpy(mm.map_off[:-1].copy()).to(dev)
    maxlab = int(mm.el.max()) if mm.el is not None and mm.el.size else 0
    b = F.DeviceBatch(len(n), mm.n_pairs, int(n.max()), int(m.max()), maxlab, 0, int(n.sum()),
                      keep["n"].data_ptr(), keep["m"].data_ptr(), keep["voff"].data_ptr(),
                      keep["eoff"].data_ptr(), keep["vl"].data_ptr(), keep["ed"].data_ptr(),
                      keep["el"].data_ptr() if keep["el"] is not None else None,
                      keep["pairs"].data_ptr(), keep["moff"].data_ptr())
    return b, keep, mm


@pytest.mark.parametrize("name", ["molecule", "dense", "wide_k"])
def test_noalloc_matches_batch_ex_twice(name):
    torch = pytest.importorskip("torch")
    if name == "molecule":
        w = W.config2(400)
    elif name == "dense":
        w = W.config3(6)
    else:   # K past the single-word packing limit: the two-word unpacked kernels
        w = W.config1(40)
        w.K = 5000
    with F.FastGED(w.cost) as g:
        ref_c, ref_m, ref_n = g.run(w)
    b, keep, mm = _device_batch(w, torch)
    for _ in range(2):
        oc = torch.full((mm.n_pairs,), -7, dtype=torch.int32, device="cuda")
        om = torch.full((int(mm.map_off[-1]),), -7, dtype=torch.int32, device="cuda")
        on = torch.full((mm.n_pairs,), -7, dtype=torch.int64, device="cuda")
        F.fastged_batch_noalloc(w.cost, b, w.K, oc.data_ptr(), om.data_ptr(), on.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert np.array_equal(oc.cpu().numpy(), ref_c)
        assert np.array_equal(om.cpu().numpy(), ref_m)
        assert np.array_equal(on.cpu().numpy(), ref_n)


def test_noalloc_rejects_batches_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    w = W.config2(4)
    b, keep, mm = _device_batch(w, torch)
    b.total_vertices = 1 << 40   # the bit-set pools alone would exceed the scratch array
    oc = torch.zeros(mm.n_pairs, dtype=torch.int32, device="cuda")
    om = torch.zeros(int(mm.map_off[-1]), dtype=torch.int32, device="cuda")
    with pytest.raises(F.FastGEDError) as ei:
        F.fastged_batch_noalloc(w.cost, b, w.K, oc.data_ptr(), om.data_ptr())
    assert ei.value.code == F.FASTGED_ERR_INVALID_ARG
