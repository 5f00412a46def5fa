"""The C-ABI library loads and exports every symbol include/flashmap.h
declares; argument checks that need no GPU behave as documented."""
import ctypes as C
import os
import re

import pytest

from paper_2609_19190_gb300 import _lib
import paper_2609_19190_gb300 as fm
from oracle import oracle as O

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "flashmap.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(fr_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = _lib.load()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(_lib.SIGNATURES), set(names) ^ set(_lib.SIGNATURES)


def test_struct_layout_matches_the_c_compiler(tmp_path):
    # offsets and sizes of the ctypes mirrors against what gcc computes
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    fields = [f for f, _ in _lib.MapParams._fields_]
    tfields = [f for f, _ in _lib.Tune._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "flashmap.h"',
           'int main(void) {', 'printf("%zu %zu\\n", sizeof(fr_map_params), sizeof(fr_tune));']
    src += ['printf("%%zu\\n", offsetof(fr_map_params, %s));' % f for f in fields]
    src += ['printf("%%zu\\n", offsetof(fr_tune, %s));' % f for f in tfields]
    src += ['return 0; }']
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.dirname(HEADER), str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(v) for v in out]
    assert sizes[0] == C.sizeof(_lib.MapParams) and sizes[1] == C.sizeof(_lib.Tune)
    offs = sizes[2:]
    assert offs[:len(fields)] == [getattr(_lib.MapParams, f).offset for f in fields]
    assert offs[len(fields):] == [getattr(_lib.Tune, f).offset for f in tfields]


def test_feature_names_and_directions_agree_with_oracle():
    assert fm.fr_feature_names() == O.feature_names()
    assert [fm.fr_direction(i) for i in range(13)] == O.directions()
    with pytest.raises(fm.FlashmapError):
        fm.fr_direction(13)


def test_params_init_defaults():
    p = fm.fr_map_params_init(10, 11, 12)
    assert (p.nx, p.ny, p.nz) == (10, 11, 12)
    assert p.disc_mode == fm.FR_FBN and p.bin_count == 16 and p.kernel_radius == 1
    assert fm.selected_features(p) == list(range(93))  # the benchmark maps by default
    q = fm.fr_map_params_init(4, 4, 4, features=[18, 19, 41], kernel_radius=3)
    assert fm.selected_features(q) == [18, 19, 41] and q.kernel_radius == 3


def test_invalid_arguments_are_rejected_without_a_device():
    L = _lib.load()
    h = C.c_void_p()
    mask = (C.c_uint8 * 8)(*([1] * 8))
    for field, value in [("kernel_radius", 0), ("kernel_radius", 8), ("bin_count", 0),
                         ("bin_count", 256), ("glcm_distance", 0), ("nx", 0),
                         ("disc_mode", 5), ("aggregation", 2)]:
        p = fm.fr_map_params_init(2, 2, 2)
        setattr(p, field, value)
        assert L.fr_map_plan(C.byref(p), mask, None, C.byref(h)) == 1, field
    p = fm.fr_map_params_init(2, 2, 2, disc_mode=fm.FR_FBW, bin_width=0.0)
    assert L.fr_map_plan(C.byref(p), mask, None, C.byref(h)) == 1
    p = fm.fr_map_params_init(2, 2, 2, features=[])
    assert L.fr_map_plan(C.byref(p), mask, None, C.byref(h)) == 1
    p = fm.fr_map_params_init(2, 2, 2)
    assert L.fr_map_plan(C.byref(p), None, None, C.byref(h)) == 1
    assert L.fr_map_run(None, None, None, None) == 1
    assert L.fr_map_sync_status(None) == 1
    L.fr_map_destroy(None)
    L.fr_batch_destroy(None)
    assert L.fr_feature_name(102) is None and L.fr_feature_count() == 101
    assert L.fr_scalar_feature_count() == 102
    assert L.fr_feature_name(101) == b"firstorder_StandardDeviation"
    # the scalar-only statistic has no map
    p = fm.fr_map_params_init(2, 2, 2, features=[0, fm.FR_SCALAR_STDDEV])
    assert L.fr_map_plan(C.byref(p), mask, None, C.byref(h)) == 1
    assert L.fr_feature_name(93) == b"firstorder_MedianAbsoluteDeviation"
    assert L.fr_status_string(3) == b"more than 255 gray levels"
