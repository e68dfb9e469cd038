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
    b = F.DeviceBatch(len(n), mm.n_pairs, int(max(n.max(), 1)), int(m.max()), maxlab, 0,
                      int(n.sum()), int(m.sum()), int(mm.map_off[-1]),
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


def _run_noalloc(w, b, mm, torch):
    """fastged_batch_noalloc on device outputs; (status, cost, map, n_evals) on the host."""
    oc = torch.full((max(mm.n_pairs, 1),), -7, dtype=torch.int32, device="cuda")
    om = torch.full((max(int(mm.map_off[-1]), 1),), -7, dtype=torch.int32, device="cuda")
    on = torch.full((max(mm.n_pairs, 1),), -7, dtype=torch.int64, device="cuda")
    try:
        F.fastged_batch_noalloc(w.cost, b, w.K, oc.data_ptr(), om.data_ptr(), on.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
        rc = F.FASTGED_OK
    except F.FastGEDError as e:
        rc = e.code
    torch.cuda.synchronize()
    return rc, oc.cpu().numpy(), om.cpu().numpy(), on.cpu().numpy()


def _bad_cases(w, mm):
    """(name, change to the device arrays or host bounds) that the device-side checks must
    reject before any kernel reads an edge or writes a map."""
    g0 = int(mm.pairs[0][0])
    return [
        ("endpoint past n", lambda k, b: k["ed"].__setitem__(0, 999)),
        ("self-loop", lambda k, b: k["ed"].__setitem__(1, int(k["ed"][0]))),
        ("pair index past n_graphs", lambda k, b: k["pairs"].__setitem__(1, 10 ** 6)),
        ("graph_n above max_n", lambda k, b: k["n"].__setitem__(g0, b.max_n + 1)),
        ("edge range past total_edges",
         lambda k, b: k["eoff"].__setitem__(g0, b.total_edges)),
        ("map past map_len", lambda k, b: k["moff"].__setitem__(0, b.map_len)),
    ]


def test_noalloc_rejects_inconsistent_device_data_and_recovers():
    """Device data that contradicts the host bounds (or is malformed) returns
    FASTGED_ERR_INVALID_ARG without reading or writing out of range; the next valid call on the
    same (shared) scratch array gives the results of fastged_batch_ex again."""
    torch = pytest.importorskip("torch")
    w = W.config2(60)
    with F.FastGED(w.cost) as g:
        ref = g.run(w)
    for name, spoil in _bad_cases(w, F.marshal(w)):
        b, keep, mm = _device_batch(w, torch)
        spoil(keep, b)
        rc, *_ = _run_noalloc(w, b, mm, torch)
        assert rc == F.FASTGED_ERR_INVALID_ARG, name
        b, keep, mm = _device_batch(w, torch)
        rc, c, m, n = _run_noalloc(w, b, mm, torch)
        assert rc == F.FASTGED_OK, name
        for x, y in zip((c, m, n), ref):
            assert np.array_equal(x, y), name


def test_noalloc_eight_label_planes_and_an_empty_batch():
    """Edge labels up to 5 (three planes, served by the eight-plane kernel), then a batch
    with no pairs (nothing to do, FASTGED_OK)."""
    torch = pytest.importorskip("torch")
    w = W.config2(80, seed=21)
    st = W.Stream(21, 5)
    for gr in w.graphs:
        gr.elabel = st.randint(0, 5, gr.m).astype(np.int32)
    with F.FastGED(w.cost) as g:
        ref = g.run(w)
    b, keep, mm = _device_batch(w, torch)
    assert b.max_elabel >= 4
    for _ in range(2):
        rc, c, m, n = _run_noalloc(w, b, mm, torch)
        assert rc == F.FASTGED_OK
        for x, y in zip((c, m, n), ref):
            assert np.array_equal(x, y)
    b.n_pairs = 0
    rc, *_ = _run_noalloc(w, b, mm, torch)
    assert rc == F.FASTGED_OK


def test_noalloc_graphs_sharing_label_rows():
    """Two graphs whose label ranges coincide (the caller stores one label array for both):
    each still gets bit-set rows of its own, so the results equal those of two separate
    copies."""
    torch = pytest.importorskip("torch")
    base = W.config2(30, seed=23)
    a = base.graphs[0]
    twin = W.Graph(a.n, a.vlabel.copy(), base.graphs[2].edges[:0].copy(), None)
    # twin: same vertices and labels as graph 0, no edges
    w = W.Workload("twins", [a, twin, base.graphs[1]],
                   np.array([[0, 2], [1, 2], [2, 0], [2, 1]], np.int32), base.cost, base.K)
    with F.FastGED(w.cost) as g:
        ref = g.run(w)
    b, keep, mm = _device_batch(w, torch)
    keep["voff"][1] = keep["voff"][0]    # graph 1 reads graph 0's label rows
    rc, c, m, n = _run_noalloc(w, b, mm, torch)
    assert rc == F.FASTGED_OK
    for x, y in zip((c, m, n), ref):
        assert np.array_equal(x, y)
