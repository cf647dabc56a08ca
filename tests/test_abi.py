"""The C-ABI library loads, exports every symbol include/usp.h declares, and
rejects invalid arguments before touching a device (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1808_03801_gb300 import usp as U
from paper_1808_03801_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "usp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(usp_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = U.lib()
    names = _declared()
    assert "usp_create" in names and "usp_step" in names and "usp_sample_macro" in names
    for n in names:
        assert hasattr(L, n), n


def test_status_strings():
    assert U.lib().usp_status_string(0) == b"ok"
    assert U.lib().usp_status_string(-4) == b"capacity exceeded"


def _create_rc(w, pipeline=None):
    gas, grid, faces, segs, nseg, params = U.make_structs(w, pipeline)
    h = ctypes.c_void_p()
    rc = U.lib().usp_create(ctypes.byref(gas), ctypes.byref(grid), faces, segs, nseg, ctypes.byref(params), None,
                            None, ctypes.byref(h))
    assert not h.value or rc == 0
    return rc


@pytest.mark.parametrize("mutate", [
    lambda w: w["params"].__setitem__("ppc_ref", 0),
    lambda w: w["grid"].__setitem__("ny", 0),
    lambda w: w["gas"].__setitem__("mass", -1.0),
    lambda w: w["params"].__setitem__("body_accel", (0.0, 1.0, 0.0)),
    lambda w: w["faces"].__setitem__(2, {"kind": "periodic", "T": 273.0, "u": (0, 0, 0), "n": 0.0}),
    lambda w: w["params"].__setitem__("mode", "bogus") if False else w["params"].__setitem__("n_avg", 0),
    lambda w: w["params"].__setitem__("precision", "fp64") or w["params"].__setitem__("pipeline", "fused"),
    lambda w: w["params"].__setitem__("dt_over_tauc", 0.0),
    lambda w: w["params"].update(flux_axis=1, flux_pos=0.5),             # no x axis in 1-D
    lambda w: w["params"].update(flux_axis=2, flux_pos=0.0),             # on a face
    lambda w: w["params"].update(flux_axis=2, flux_pos=1.0),             # outside the domain
    lambda w: w["params"].update(flux_axis=3, flux_pos=1e-7),
])
def test_invalid_arguments_rejected_without_gpu(mutate):
    w = W.couette(ny=10, ppc=10)
    mutate(w)
    assert _create_rc(w) == -1


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of the public structs have the C compiler's sizes
    and field offsets, and the binding's USP_NEXT_PID_AUTO is the header's
    (include/usp.h compiled as plain C)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"usp_gas": U.Gas, "usp_grid": U.Grid, "usp_bc": U.Bc, "usp_wall_segment": U.WallSegment,
               "usp_params": U.Params, "usp_region": U.Region, "usp_allocator": U.Allocator,
               "usp_info": U.Info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "usp.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines.append('printf("USP_NEXT_PID_AUTO value %u\\n", USP_NEXT_PID_AUTO);')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    assert got[("USP_NEXT_PID_AUTO", "value")] == U.NEXT_PID_AUTO
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])


@pytest.mark.parametrize("pipeline", ["plain", "fused"])
@pytest.mark.parametrize("key", ["selection", "es_sampler"])
def test_ablation_codes_out_of_range_rejected(pipeline, key):
    """Both pipelines run fixed-count selection and the Gallis-Torczynski
    sampler; a code outside USP_SELECT_* / USP_SAMPLER_* is INVALID_ARG."""
    w = W.sod(ny=10, ppc_left=10)
    w["params"]["pipeline"] = pipeline
    if pipeline == "fused":
        w = W.with_precision(w, "fp32")
    gas, grid, faces, segs, nseg, params = U.make_structs(w, pipeline)
    setattr(params, key, 2)
    h = ctypes.c_void_p()
    rc = U.lib().usp_create(ctypes.byref(gas), ctypes.byref(grid), faces, segs, nseg, ctypes.byref(params), None,
                            None, ctypes.byref(h))
    assert rc == -1 and not h.value


@pytest.mark.parametrize("change", [
    dict(pipeline="fused", precision="fp32"),   # weighted particles: plain FP64 only
    dict(r_p=0.0),                              # Eq. 25 needs r_p > 0
    dict(selection="fixed_count"),              # the default selection and sampler only
    dict(slab_count=2),                         # one domain
])
def test_weighted_options_validated_before_any_device_work(change):
    w = W.couette(ny=10, ppc=10, precision="fp64")
    w["params"].update(weighted=1)
    w["params"].update(change)
    assert _create_rc(w) == -1


def test_weighted_particles_reject_reservoir_faces():
    w = W.slit(nx=20, ny=10, ppc=5, precision="fp64")
    w["params"].update(weighted=1, pipeline="plain")
    assert _create_rc(w) == -1
