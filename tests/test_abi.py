"""The C-ABI library builds, loads and exports every entry point include/dem.h declares
(no GPU needed: nothing here calls into the device)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "dem.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dem_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("dem_world_create", "dem_add_material", "dem_add_box_walls", "dem_add_clump_template",
                 "dem_add_clumps", "dem_initialize", "dem_step", "dem_get_owner_state", "dem_get_contacts",
                 "dem_save_state", "dem_batch_step", "dem_schedule_train", "dem_get_diagnostics"):
        assert must in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2311_04648_gb300 import build as b
    lib = b.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (dem_[a-z0-9_]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_sets_every_signature():
    from paper_2311_04648_gb300 import dem
    try:
        L = dem.load()
    except OSError as e:      # e.g. no CUDA runtime library on this host
        pytest.skip(f"cannot load the CUDA runtime here: {e}")
    for n in declared_functions():
        f = getattr(L, n)
        assert f.restype is not None


def test_calls_without_a_device_fail_cleanly():
    import ctypes as C
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except Exception:
        pass
    from paper_2311_04648_gb300 import dem
    try:
        L = dem.load()
    except OSError as e:
        pytest.skip(f"cannot load the CUDA runtime here: {e}")
    d = dem.WorldDesc()
    for a in range(3):
        d.box_hi[a] = 1.0
    h = C.c_void_p()
    st = L.dem_world_create(C.byref(d), C.byref(h))
    assert st == dem.ERR_CUDA
    assert b"device" in L.dem_last_error(None)
    # argument validation needs no device
    st = L.dem_world_create(None, C.byref(h))
    assert st == dem.ERR_ARG


def test_smoke_scene_builds_and_has_contacts():
    import __graft_entry__ as g
    import oracle

    s = g.smoke_scene()
    o = oracle.OracleWorld(s)
    assert o.step(5) == 0
    assert len(o.eval()[2]) > 100


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes mirrors of the header's structs have the C sizes and field offsets (the
    header compiled as C99 by gcc prints them)."""
    import ctypes
    import shutil
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2311_04648_gb300 import dem
    mirrors = {"dem_world_desc": dem.WorldDesc, "dem_stats": dem.Stats, "dem_tuning": dem.Tuning,
               "dem_diagnostics": dem.Diagnostics}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dem.h"', "int main(void) {"]
    for cname, cls in mirrors.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
