"""The C-ABI library loads and exports every function include/o2tpc.h declares
(no GPU needed: nothing is called that touches a device)."""
import ctypes
import os
import re

from paper_2106_03636_gb300 import _build, o2tpc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "o2tpc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s+(o2tpc_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("o2tpc_create", "o2tpc_submit_tf", "o2tpc_submit_many", "o2tpc_poll", "o2tpc_destroy", "o2tpc_result_release",
              "o2tpc_strerror", "o2tpc_get_stage", "o2tpc_get_tuning"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_build.build_tpc())
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_strerror_without_gpu():
    assert o2tpc.o2tpc_strerror(o2tpc.O2TPC_ETOOBIG).startswith("time frame")
    assert o2tpc.o2tpc_strerror(12345) == "unknown status"


def test_binding_structures_match_header_sizes():
    # 64-bit layout of the C structs as the header defines them
    assert ctypes.sizeof(o2tpc.o2tpc_tf) == 8 + 4 + 4 + 6 * 8 + 8 + 8 + 8
    assert ctypes.sizeof(o2tpc.o2tpc_stats) == 5 * 8 + 4 * 4 + 8 + 18 * 4 + 2 * 4
    # device, budget, inflight, batch, bz, vdrift, flags(+pad), 2 callbacks, user, stream, batch_full,
    # two launch shapes, graph clusters, graph TFs + nf_staged, cache path, debug_inject(+pad)
    assert ctypes.sizeof(o2tpc.o2tpc_config) == 8 + 8 + 4 + 4 + 8 + 8 + 8 + 8 * 4 + 8 + 4 + 4 + 8 + 8 + 8 + 8
    assert ctypes.sizeof(o2tpc.o2tpc_tuning) == 5 * 4 + 9 * 4


def test_binding_layout_matches_the_compiled_header(tmp_path):
    """sizeof / offsetof of every public struct, from the header compiled by
    gcc, against the ctypes mirror."""
    import subprocess

    structs = {"o2tpc_tf": o2tpc.o2tpc_tf, "o2tpc_stats": o2tpc.o2tpc_stats, "o2tpc_result": o2tpc.o2tpc_result,
               "o2tpc_config": o2tpc.o2tpc_config, "o2tpc_tuning": o2tpc.o2tpc_tuning,
               "o2tpc_digits": o2tpc.o2tpc_digits, "o2tpc_ctf_clusters": o2tpc.o2tpc_ctf_clusters}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "o2tpc.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split("\n")
               if line)
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"
