"""CPU checks of the C ABI: the library builds for sm_103a, loads without a
GPU, and exports exactly the entry points that include/sell.h declares; the
Python binding names the same set.  No compute call is made."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sell.h")).read()
    return set(re.findall(r"^SELL_API\s+[\w\s\*]+?\b(sell_\w+)\s*\(", src, flags=re.M))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1307_6209_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("sell_build", "sell_spmv", "sell_spmmv", "sell_free", "sell_info", "sell_export",
                 "sell_batch_create", "sell_batch_run", "sell_batch_free", "sell_set_allocator"):
        assert name in d


def test_library_exports_exactly_the_header(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.split() and ln.split()[-1].startswith("sell_")}
    assert exported == _declared()


def test_library_loads_and_binding_covers_every_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name)
    from paper_1307_6209_gb300 import sell
    assert set(sell.SIGNATURES) == _declared()
    sell.load()
    assert sell.sell_strerror(sell.SELL_EINVAL) == "invalid argument"


def test_struct_layouts_match_header(lib_path):
    """Compile a tiny C program against sell.h that prints the struct sizes and
    offsets, and compare with the ctypes mirrors."""
    from paper_1307_6209_gb300 import sell
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "sell.h"
int main(void){
 printf("%zu %zu %zu %zu\n", sizeof(sell_csr), sizeof(sell_opts), sizeof(sell_info_t), sizeof(sell_batch_item));
 printf("%zu %zu %zu %zu\n", offsetof(sell_csr,val_type), offsetof(sell_opts,flags), offsetof(sell_info_t,beta), offsetof(sell_batch_item,k));
 return 0;}
"""
    d = os.path.join(ROOT, "paper_1307_6209_gb300", "_build")
    os.makedirs(d, exist_ok=True)
    c = os.path.join(d, "layout.c")
    exe = os.path.join(d, "layout")
    open(c, "w").write(prog)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = list(map(int, lines[0].split()))
    offs = list(map(int, lines[1].split()))
    assert sizes == [ctypes.sizeof(sell.sell_csr), ctypes.sizeof(sell.sell_opts),
                     ctypes.sizeof(sell.sell_info_t), ctypes.sizeof(sell.sell_batch_item)]
    assert offs == [sell.sell_csr.val_type.offset, sell.sell_opts.flags.offset,
                    sell.sell_info_t.beta.offset, sell.sell_batch_item.k.offset]


def test_every_struct_field_matches_header(lib_path, tmp_path):
    """Every field of every ctypes mirror against offsetof() in C, plus the
    sizes: a layout slip would pass wrong arguments silently."""
    from paper_1307_6209_gb300 import sell
    mirrors = [sell.sell_csr, sell.sell_opts, sell.sell_info_t, sell.sell_batch_item, sell.sell_server_opts,
               sell.sell_request_info, sell.sell_server_stats_t]
    body, want = [], []
    for m in mirrors:
        body.append(f'printf("%zu\\n", sizeof({m.__name__}));')
        want.append(ctypes.sizeof(m))
        for name, _ in m._fields_:
            body.append(f'printf("%zu\\n", offsetof({m.__name__}, {name}));')
            want.append(getattr(m, name).offset)
    prog = "#include <stdio.h>\n#include <stddef.h>\n#include \"sell.h\"\nint main(void){\n" + \
        "\n".join(body) + "\nreturn 0;}\n"
    c, exe = tmp_path / "fields.c", tmp_path / "fields"
    c.write_text(prog)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(c), "-o",
                    str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    assert got == want
