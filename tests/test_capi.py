"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
and exports every function include/bchar.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bchar.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bchar_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("bchar_create_mesh", "bchar_set_velocity", "bchar_step", "bchar_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1908_05834_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_marshals_options_and_status_strings():
    from paper_1908_05834_gb300 import build
    build.build()
    from paper_1908_05834_gb300 import bchar
    o = bchar.default_options()
    assert (o.balls_per_axis, o.n_scale, o.precision) == (2, 10, bchar.FP64)
    assert o.penalty == pytest.approx(1e-7) and o.qp_tol == pytest.approx(1e-9)
    # the last fields: a mismatch between the ctypes mirror and the header would show here
    assert (o.qp_precond, o.qp_warm_start) == (1, 1)
    assert bchar.bchar_status_string(0) == b"ok"
    assert b"boundary" in bchar.bchar_status_string(4)


def test_footprint_estimate_on_the_host():
    """bchar_estimate_device_bytes needs no GPU: it grows with the mesh, counts
    the tight ball packing of stretched cells, and rejects bad arguments."""
    from paper_1908_05834_gb300 import build
    build.build()
    import numpy as np
    from paper_1908_05834_gb300 import bchar, inputs
    u = [inputs.uniform_coords(64)] * 2
    e64 = bchar.estimate_device_bytes(u)
    e128 = bchar.estimate_device_bytes([inputs.uniform_coords(128)] * 2)
    assert 3.5 < e128 / e64 < 4.5  # ~ proportional to the cells
    rng = np.random.Generator(np.random.PCG64(1))
    s = [inputs.stretched_coords(rng, 64, 0.5, 1.5), inputs.stretched_coords(rng, 64, 0.5, 1.5)]
    assert bchar.estimate_device_bytes(s) > e64  # stretched cells hold more balls
    e3 = bchar.estimate_device_bytes([inputs.uniform_coords(16)] * 3)
    assert e3 > 16 ** 3 * 1000
    with pytest.raises(bchar.BcharError):
        bchar.estimate_device_bytes(u, bchar.default_options(qp_warm_start=2))
    with pytest.raises(bchar.BcharError):
        bchar.estimate_device_bytes([np.array([0.0, 0.5, 0.5, 1.0])] * 2)  # a zero width


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of bchar_options and bchar_step_info have the
    header's field names, offsets and sizes (a C program compiled against
    include/bchar.h prints them); bchar_step_batch indexes an array of
    bchar_step_info, so a size mismatch would shift every instance's info."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1908_05834_gb300 import bchar
    pairs = (("bchar_options", bchar.Options), ("bchar_step_info", bchar.StepInfo))
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "bchar.h"', "int main(void) {"]
    for cname, cls in pairs:
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'    printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line}
    for cname, cls in pairs:
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
