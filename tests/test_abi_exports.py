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


_HANDLES = {"sell_handle", "sell_batch_plan", "sell_server_t", "sell_alloc_fn", "sell_free_fn"}
_SCALARS = {"int32_t": ("i", 4), "sell_status": ("i", 4), "int64_t": ("i", 8), "uint32_t": ("u", 4),
            "uint64_t": ("u", 8), "size_t": ("u", 8), "double": ("f", 8)}


def _c_kind(t):
    t = " ".join(t.replace("const", " ").split())
    if "*" in t or t in _HANDLES:
        return ("p", 8)
    return _SCALARS[t]


def _ctypes_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, (ctypes._Pointer, ctypes._CFuncPtr)):
        return ("p", 8)
    if t is ctypes.c_double:
        return ("f", 8)
    return ("i" if t(-1).value < 0 else "u", ctypes.sizeof(t))


def test_binding_argument_types_match_prototypes():
    """Each ctypes signature of the binding against the prototype in
    include/sell.h: the same number of arguments, each of the same kind and
    width (a 32-bit integer where the C side reads 64 bits would corrupt the
    call silently), and pointers to the struct mirrors of the named types."""
    from paper_1307_6209_gb300 import sell
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "sell.h")).read(), flags=re.S)
    protos = {m.group(2): (m.group(1), m.group(3)) for m in
              re.finditer(r"SELL_API\s+([\w\s\*]+?)\b(sell_\w+)\s*\(([^;]*?)\)\s*;", src, flags=re.S)}
    assert set(protos) == set(sell.SIGNATURES)
    for name, (ret, params) in protos.items():
        res, args = sell.SIGNATURES[name]
        assert _c_kind(ret) == _ctypes_kind(res), name
        ps = [] if params.strip() == "void" else [p.strip() for p in params.split(",")]
        assert len(ps) == len(args), name
        for p, a in zip(ps, args):
            ctype = re.sub(r"\b\w+\s*$", "", p).strip()  # drop the parameter name
            assert _c_kind(ctype) == _ctypes_kind(a), f"{name}: {p}"
            base = " ".join(ctype.replace("const", " ").replace("*", " ").split())
            if ctype.count("*") == 1 and hasattr(sell, base) and isinstance(getattr(sell, base), type) \
                    and issubclass(getattr(sell, base), ctypes.Structure):
                assert issubclass(a, ctypes._Pointer) and a._type_ is getattr(sell, base), f"{name}: {p}"


def test_c_program_links_and_calls_host_only_entry_points(lib_path, tmp_path):
    """A C program that takes the address of every declared entry point links
    against the library, and runs the calls that need no GPU: error strings,
    argument validation before any device work, the allocator hook."""
    names = sorted(_declared())
    prog = ["#include <stdio.h>", "#include <string.h>", '#include "sell.h"',
            "static void *fake_alloc(size_t n, void *c, void *s) { (void)n; (void)c; (void)s; return 0; }",
            "static void fake_free(void *p, void *c, void *s) { (void)p; (void)c; (void)s; }",
            "int main(void) {", "  void *fns[] = {"]
    prog += [f"    (void *)&{n}," for n in names]
    prog += ["  };",
             "  int missing = 0;",
             "  for (size_t i = 0; i < sizeof fns / sizeof fns[0]; ++i) missing += fns[i] == 0;",
             "  if (missing) return 2;",
             '  if (strcmp(sell_strerror(SELL_EINVAL), "invalid argument")) return 3;',
             "  if (sell_build(NULL, NULL, NULL, NULL) != SELL_EINVAL) return 4;",
             "  if (sell_spmv(NULL, NULL, NULL, 0, NULL) != SELL_EINVAL) return 5;",
             "  if (strlen(sell_last_error()) == 0) return 6;",
             "  if (sell_set_allocator(fake_alloc, NULL, NULL) != SELL_EINVAL) return 7;",
             "  if (sell_set_allocator(fake_alloc, fake_free, NULL) != SELL_OK) return 8;",
             "  if (sell_set_allocator(NULL, NULL, NULL) != SELL_OK) return 9;",
             "  if (sell_free(NULL) != SELL_OK || sell_server_destroy(NULL) != SELL_OK) return 10;",
             '  printf("ok %zu\\n", sizeof fns / sizeof fns[0]);',
             "  return 0;", "}"]
    c, exe = tmp_path / "use.c", tmp_path / "use"
    c.write_text("\n".join(prog) + "\n")
    libdir = os.path.dirname(lib_path)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(c),
                    "-L", libdir, "-lsellcs", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip() == f"ok {len(names)}"
