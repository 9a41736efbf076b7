"""The ctypes binding's structures against the C headers, on the CPU.

Every `typedef struct { ... } name;` of include/*.h is compiled by the host C
compiler into a small program that prints sizeof and the offset of each field;
the binding's ctypes class of the same name must list the same fields, in the
same order, at the same offsets, with the same total size.  A field added to a
header but not to the binding (or the other way round) fails here instead of
corrupting arguments at run time."""
import ctypes
import keyword
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def _structs():
    """(struct name, [field names]) of every typedef'd struct in include/*.h."""
    out = []
    for h in sorted(os.listdir(INCLUDE)):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(INCLUDE, h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"typedef\s+struct\s*\w*\s*\{(.*?)\}\s*(\w+)\s*;", src, flags=re.S):
            names = []
            for decl in m.group(1).split(";"):
                decl = " ".join(decl.split())
                if not decl:
                    continue
                # "type a, *b, c[3]": the declarators after the type words
                first = re.match(r"((?:const\s+)?(?:unsigned\s+)?\w+)\s*(.*)$", decl)
                for d in first.group(2).split(","):
                    nm = re.search(r"(\w+)\s*(\[[^\]]*\])?\s*$", d.strip())
                    names.append(nm.group(1))
            out.append((m.group(2), names))
    return out


def _c_layout(tmp_path, structs):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>"]
    lines += [f'#include "{h}"' for h in sorted(os.listdir(INCLUDE)) if h.endswith(".h")]
    lines.append("int main(void) {")
    for name, fields in structs:
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    res = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in res.splitlines():
        name, field, value = line.split()
        layout[(name, field)] = int(value)
    return layout


def test_binding_structs_match_the_headers(tmp_path):
    from paper_1501_06211_gb300 import ddel
    structs = _structs()
    assert len(structs) >= 10
    layout = _c_layout(tmp_path, structs)
    checked = 0
    for name, fields in structs:
        cls = getattr(ddel, name, None)
        assert cls is not None, f"the binding has no structure {name}"
        # a C field named like a Python keyword carries a trailing underscore
        py = [f[0] for f in cls._fields_]
        cname = [n[:-1] if n.endswith("_") and keyword.iskeyword(n[:-1]) else n for n in py]
        assert cname == fields, (name, cname, fields)
        for p, f in zip(py, fields):
            assert getattr(cls, p).offset == layout[(name, f)], (name, f)
        assert ctypes.sizeof(cls) == layout[(name, "size")], name
        checked += 1
    assert checked == len(structs)
