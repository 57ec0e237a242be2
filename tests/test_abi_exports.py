"""The C-ABI library builds, loads without a GPU and exports every function
that include/damn.h declares; the Python binding carries the same names.
Only calls that do no device work are made here (version, size queries,
argument checks that fail before any CUDA call)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "damn.h")


def declared_structs():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"}\s*(damn_\w+)\s*;", text)))


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(damn_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2307_06305_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_parses():
    names = declared_functions()
    assert len(names) >= 30
    for must in ("damn_csr_to_dacsr", "damn_spmv_dacsr16", "damn_spmv_csr32", "damn_rcm_order",
                 "damn_permute_sym", "damn_cg", "damn_cg_ir", "damn_spmm_dacsr16",
                 "damn_batch_plan_create", "damn_plan_autotune", "damn_csr_to_dacsr_noalloc"):
        assert must in names


def test_every_declared_symbol_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(lib):
    from paper_2307_06305_gb300 import damn
    declared = set(declared_functions())
    bound = {n for n in dir(damn) if n.startswith("damn_") and callable(getattr(damn, n))
             and not isinstance(getattr(damn, n), type)}
    assert bound <= declared, bound - declared
    for n in ("damn_csr_to_dacsr", "damn_csr_to_dacsr_noalloc", "damn_spmv_dacsr16",
              "damn_spmv_csr32", "damn_rcm_order", "damn_permute_sym", "damn_rcm_permute",
              "damn_cg", "damn_cg_ir", "damn_spmm_dacsr16"):
        assert n in bound


def test_host_only_calls(lib):
    lib.damn_version.restype = ctypes.c_int
    assert lib.damn_version() >= 100
    lib.damn_permute_sym_workspace_size.restype = ctypes.c_size_t
    lib.damn_permute_sym_workspace_size.argtypes = [ctypes.c_int32]
    assert lib.damn_permute_sym_workspace_size(1 << 20) >= 4 * (1 << 20)
    lib.damn_cg_workspace_size.restype = ctypes.c_size_t
    lib.damn_cg_workspace_size.argtypes = [ctypes.c_int32]
    assert lib.damn_cg_workspace_size(1000) >= 3 * 8 * 1000
    # argument checks return before touching a device
    lib.damn_plan_create.restype = ctypes.c_int
    P = ctypes.c_void_p
    lib.damn_plan_create.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, P, ctypes.c_int,
                                     P, ctypes.c_int, P, ctypes.POINTER(P)]
    out = P()
    assert lib.damn_plan_create(-1, 4, 0, None, 1, None, 0, None, ctypes.byref(out)) == -1
    lib.damn_last_error.restype = ctypes.c_char_p
    assert lib.damn_last_error()


def test_struct_layouts_match_c(tmp_path):
    """Every struct the binding mirrors has the C compiler's size and field
    offsets (the header is compiled as plain C)."""
    import subprocess
    from paper_2307_06305_gb300 import damn
    structs = declared_structs()
    mirrored = [s for s in structs if hasattr(damn, s)]
    assert set(mirrored) >= {"damn_fit_info", "damn_plan_desc", "damn_cg_result", "damn_mat_desc",
                             "damn_batch_desc", "damn_bw_info"}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "damn.h"', "int main(void) {"]
    for s in mirrored:
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for f, _ in getattr(damn, s)._fields_:
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for s in mirrored:
        cls = getattr(damn, s)
        assert ctypes.sizeof(cls) == c[(s, "size")], s
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == c[(s, f)], (s, f)


def test_plain_c_program_links_and_calls(tmp_path):
    """A plain C program (no C++, no Python) includes damn.h, links
    libdamn.so and calls host-side entry points: the library is usable
    through its C ABI alone."""
    import subprocess
    from paper_2307_06305_gb300 import build
    path = build.build()
    src = tmp_path / "use_damn.c"
    src.write_text(r"""
#include <stdio.h>
#include <stdint.h>
#include "damn.h"
int main(void) {
  /* path 0-1-2-3-4 relabelled as 2-0-4-1-3 (diagonal entries included) */
  const int32_t rowptr[6] = {0, 3, 6, 8, 10, 13};
  const int32_t col[13] = {0, 2, 4, 1, 3, 4, 0, 2, 1, 3, 0, 1, 4};
  int32_t perm[5];
  int64_t wb = -1, wa = -1;
  int rc = damn_rcm_order(5, 13, rowptr, col, perm, &wb, &wa);
  if (rc != DAMN_OK) { printf("rcm rc %d %s\n", rc, damn_last_error()); return 1; }
  printf("perm %d %d %d %d %d w %lld %lld\n", perm[0], perm[1], perm[2], perm[3], perm[4],
         (long long)wb, (long long)wa);
  rc = damn_spmv_dacsr16(-1, 1, 0, NULL, NULL, NULL, DAMN_F64, NULL, NULL, 1.0, 0.0, NULL, NULL);
  printf("spmv rc %d %s\n", rc, damn_last_error());
  printf("version %d\n", damn_version());
  return rc == DAMN_ERR_INVALID_ARG ? 0 : 2;
}
""")
    exe = tmp_path / "use_damn"
    libdir = os.path.dirname(path)
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-ldamn", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    lines = out.stdout.splitlines()
    # the hand-worked RCM of this path (tests/golden/rcm_hand_examples.txt)
    # numbers it along the path: bandwidth 4 before, 1 after
    assert lines[0] == "perm 3 1 4 0 2 w 4 1", lines[0]
    assert lines[1].startswith("spmv rc -1 damn_spmv_dacsr16")
