"""The C-ABI library loads and exports every entry point declared in include/*.h.

No compute calls: these run without a GPU.
"""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        for m in re.finditer(r"NRRS_API\s+[\w\s\*]+?\b(nrrs_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_header_declares_the_abi():
    names = _declared()
    for n in ("nrrs_create_scene", "nrrs_render", "nrrs_query_factors", "nrrs_destroy_scene",
              "nrrs_status_string", "nrrs_split", "nrrs_normalize"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2510_07868_b300 import build

    lib_path = build.build()
    import ctypes

    lib = ctypes.CDLL(lib_path)
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2510_07868_b300 import nrrs

    assert set(nrrs.EXPORTED) == _declared()
    for name in nrrs.EXPORTED:
        assert callable(getattr(nrrs, name))


def test_status_strings_without_gpu():
    from paper_2510_07868_b300 import nrrs

    assert nrrs.nrrs_status_string(0) == "ok"
    assert nrrs.nrrs_status_string(1) == "invalid argument"
    assert nrrs.nrrs_status_string(99) == "unknown status"


def test_struct_layouts_match_header():
    import ctypes

    from paper_2510_07868_b300 import inputs, nrrs

    assert ctypes.sizeof(nrrs.RenderOpts) == 128
    assert ctypes.sizeof(nrrs.RenderStats) == 32 * (8 + 8 + 4 + 8 + 8 + 8) + 4 * 8 + 8 + 96
    assert inputs.MATERIAL_DTYPE.itemsize == 40 and inputs.CAMERA_DTYPE.itemsize == 40


def test_invalid_arguments_are_rejected_without_gpu():
    from paper_2510_07868_b300 import nrrs

    with pytest.raises(nrrs.NrrsError) as e:
        nrrs.nrrs_render(None, 8, 8, 1, 4, 0, None, 0, stream=0)
    assert e.value.code == 1
    with pytest.raises(nrrs.NrrsError) as e:
        nrrs.nrrs_query_factors(None, 0, -1, 32, 0, stream=0)
    assert e.value.code == 1


def test_struct_offsets_match_the_c_compiler(tmp_path):
    """Every ctypes mirror of a header struct has the C compiler's size and field
    offsets (gcc on include/nrrs.h)."""
    import ctypes
    import subprocess

    from paper_2510_07868_b300 import nrrs

    pairs = {"nrrs_render_opts": nrrs.RenderOpts, "nrrs_render_stats": nrrs.RenderStats,
             "nrrs_train_opts": nrrs.TrainOpts, "nrrs_train_stats": nrrs.TrainStats,
             "nrrs_mixdepth_opts": nrrs.MixDepthOpts,
             "nrrs_mixdepth_result": nrrs.MixDepthResult, "nrrs_tune_report": nrrs.TuneReport,
             "nrrs_job": nrrs.Job}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "nrrs.h"', "int main(void) {"]
    expect = []
    for cname, cls in pairs.items():
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        expect.append(ctypes.sizeof(cls))
        for fname, *_ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {fname}));')
            expect.append(getattr(cls, fname).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got == expect
