"""The C ABI library builds for sm_103a, loads, and exports every function
include/fsp.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1206_4973_gb300 import build as fsp_build
from paper_1206_4973_gb300 import fsp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fsp.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(fsp_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    path = fsp_build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("fsp_create_instance", "fsp_bound_pool", "fsp_solve"):
        assert must in names
    assert set(names) == set(fsp.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_loads_and_pure_host_calls_work(lib):
    L = fsp.load()
    assert fsp.fsp_node_stride(20) == 32
    assert fsp.fsp_node_stride(15) == 16
    assert fsp.fsp_node_stride(100) == 112
    o = fsp.fsp_options()
    assert L.fsp_default_options(ctypes.byref(o)) == 0 and o.pool_size == 1024


def test_create_instance_rejects_bad_shapes_without_touching_the_device(lib):
    import numpy as np
    for p in (np.zeros((3, 1), np.int32) + 1, np.zeros((256, 3), np.int32) + 1,
              np.zeros((3, 65), np.int32) + 1, np.array([[1, 0], [2, 3]], np.int32),
              np.array([[1, 40000], [2, 3]], np.int32)):
        with pytest.raises(fsp.FspError) as e:
            fsp.fsp_create_instance(p)
        assert e.value.code == fsp.ERR_ARG


def test_library_is_built_for_sm_103a_only():
    # the build passes exactly one -gencode (sm_103a) to every nvcc call
    assert fsp_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structs have the header's sizes and offsets."""
    import subprocess
    src = tmp_path / "layout.c"
    classes = {"fsp_options": fsp.fsp_options, "fsp_stats": fsp.fsp_stats,
               "fsp_batch_result": fsp.fsp_batch_result, "fsp_batch_class_info": fsp.fsp_batch_class_info}
    fields = {st: [f for f, _ in cls._fields_] for st, cls in classes.items()}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fsp.h"', "int main(void){"]
    for st, fl in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fl:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split("\n") if l)
    for st, cls in classes.items():
        assert int(out[st]) == ctypes.sizeof(cls), st
        for f in fields[st]:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, f"{st}.{f}"
