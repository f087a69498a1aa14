"""The in-tree build's staleness check: the library counts as up to date only when it is newer
than every source the translation units include -- the .cu files, the .cuh and .h headers and
the .inc parts of fwi_api.cu -- so editing any of them rebuilds it (checked through mtimes on
a stand-in library file, without compiling)."""
import os
import re

from paper_1804_01184_gb300 import build as B


def included_files():
    """Every file named by an #include "..." in the library's sources, transitively."""
    seen, todo = set(), list(B.SOURCES)
    while todo:
        p = os.path.realpath(todo.pop())
        if p in seen:
            continue
        seen.add(p)
        for m in re.finditer(r'#include\s+"([^"]+)"', open(p).read()):
            todo.append(os.path.join(os.path.dirname(p), m.group(1)))
    return seen


def test_every_included_file_is_a_dependency():
    deps = {os.path.realpath(p) for p in B.DEPS}
    inc = included_files()
    assert any(p.endswith(".inc") for p in inc)
    assert inc <= deps, sorted(inc - deps)


def test_touching_an_inc_part_makes_the_library_stale(tmp_path, monkeypatch):
    lib = tmp_path / "libfwi.so"
    lib.write_bytes(b"")
    monkeypatch.setattr(B, "LIB", str(lib))
    newest = max(os.path.getmtime(p) for p in B.DEPS)
    os.utime(lib, (newest + 10, newest + 10))
    assert B.up_to_date()
    inc = [p for p in B.DEPS if p.endswith(".inc")]
    assert inc
    for p in inc:
        t = os.path.getmtime(p)
        os.utime(lib, (t - 10, t - 10))          # the library is older than this part
        assert not B.up_to_date(), p
