"""CPU-only checks of the C-ABI library: it builds, loads, exports every function the
header declares, and the Python mirror structs match the C layouts."""
import ctypes
import os
import re
import subprocess

from paper_2605_00830_gb300 import build as B
from paper_2605_00830_gb300 import fastged as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fastged.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fastged_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    path = B.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "fastged_batch" in names and "fastged_create" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) <= set(F.EXPORTED + [n for n in names if n.startswith("fastged_serve")]
                             + [n for n in names if n.startswith("fastged_noalloc")])


def test_version():
    assert F.fastged_version() == 10000


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "fastged.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n",'
                    'sizeof(fastged_cost_model), sizeof(fastged_graph), sizeof(fastged_pair_list),'
                    'sizeof(fastged_options), sizeof(fastged_plan_stats),'
                    'offsetof(fastged_graph, elabel), offsetof(fastged_options, use_cuda_graph));'
                    'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(prog),
                           "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(F.CostModel), ctypes.sizeof(F.GraphC), ctypes.sizeof(F.PairList),
            ctypes.sizeof(F.Options), ctypes.sizeof(F.PlanStats),
            F.GraphC.elabel.offset, F.Options.use_cuda_graph.offset]
    assert got == want


def test_header_compiles_as_c_and_cxx(tmp_path):
    for lang, comp in (("c", "gcc"), ("c++", "g++")):
        src = tmp_path / f"h.{ 'c' if lang == 'c' else 'cpp'}"
        src.write_text('#include "fastged.h"\nint (*fp)(void) = fastged_version;\nint main(void){return fp == (int (*)(void))0;}\n')
        subprocess.check_call([comp, "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                               "-c", str(src), "-o", str(tmp_path / f"h_{lang}.o")])


def test_marshalling_offsets():
    from paper_2605_00830_gb300 import workloads as W
    w = W.config2(50)
    mm = F.marshal(w)
    assert mm.n_pairs == 50
    assert int(mm.map_off[-1]) == sum(w.graphs[int(a)].n for a, _ in w.pairs)
    # the struct for graph 7 points at its own labels and edges
    g = w.graphs[7]
    addr = int(mm.gs["vlabel"][7])
    buf = (ctypes.c_int32 * g.n).from_address(addr)
    assert list(buf) == list(g.vlabel)
    addr = int(mm.gs["edges"][7])
    buf = (ctypes.c_int32 * (2 * g.m)).from_address(addr)
    assert list(buf) == list(g.edges.reshape(-1))


def test_host_entry_points_called_from_c(tmp_path):
    """A C program linked against the library calls the host-only entry points (edit path,
    partial application, fault-argument checks, error strings) on a hand-worked example."""
    path = B.build()
    prog = tmp_path / "use.c"
    prog.write_text(r'''
#include <stdio.h>
#include "fastged.h"
int main(void) {
    const int32_t vl1[3] = {0, 1, 2}, ed1[4] = {0, 1, 1, 2}, el1[2] = {0, 1};
    const int32_t vl2[3] = {0, 1, 1}, ed2[4] = {0, 1, 0, 2}, el2[2] = {1, 0};
    fastged_graph g1 = {3, vl1, 2, ed1, el1}, g2 = {3, vl2, 2, ed2, el2};
    fastged_cost_model c = {2, 4, 4, 1, 2, 2};
    const int32_t map[3] = {0, 1, -1};
    fastged_edit_op ops[16];
    int32_t n = 0;
    int64_t tot = 0;
    if (fastged_edit_path(&c, &g1, &g2, map, ops, 16, &n, &tot) != FASTGED_OK) return 1;
    printf("ops %d total %lld kinds", n, (long long)tot);
    for (int k = 0; k < n; ++k) printf(" %d", ops[k].kind);
    int32_t on = 0, om = 0, vl[6], ed[8], el[4];
    if (fastged_apply_edit_ops(&g1, &g2, map, ops, n, &on, vl, &om, ed, el) != FASTGED_OK) return 2;
    printf(" | applied n %d m %d", on, om);
    const int32_t bad[3] = {0, 0, -1};
    const int rc = fastged_edit_path(&c, &g1, &g2, bad, NULL, 0, &n, NULL);
    printf(" | bad map %d (%s)", rc, fastged_last_error(NULL) ? "msg" : "none");
    printf(" | inject %d %d\n", fastged_inject_fault(7, 1), fastged_inject_fault(0, 0));
    return 0;
}
''')
    exe = tmp_path / "use"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(prog),
                           path, "-o", str(exe), f"-Wl,-rpath,{os.path.dirname(path)}"])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ("ops 5 total 13 kinds 0 2 3 4 5 | applied n 3 m 2 | "
                                  f"bad map {F.FASTGED_ERR_INVALID_ARG} (msg) | "
                                  f"inject {F.FASTGED_ERR_INVALID_ARG} 0")
