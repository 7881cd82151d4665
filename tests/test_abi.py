"""Host-side checks of the C ABI (no GPU): the library loads, exports every function
declared in include/gwc.h, the binding's struct layouts match the header, and calls
made without a device fail with a status instead of crashing."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g():
    from paper_2605_23538_gb300 import build
    build.build()
    import paper_2605_23538_gb300 as g
    g.lib()
    return g


def header_functions():
    src = open(os.path.join(ROOT, "include", "gwc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gwc_\w+)\s*\(", src)))


def test_exports_every_declared_function(g):
    declared = header_functions()
    assert len(declared) >= 10
    import ctypes
    lib = ctypes.CDLL(g.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(g.EXPORTS) == declared


STRUCTS = {"Events": "gwc_events", "Los": "gwc_los", "Injections": "gwc_injections",
           "Options": "gwc_options", "Info": "gwc_info", "TuneResult": "gwc_tune_result",
           "KdeOptions": "gwc_kde_options"}


def test_struct_layouts_match_the_compiled_header(g, tmp_path):
    # a C program compiled against include/gwc.h prints each struct's size and the offset
    # of every field the binding declares; the ctypes layouts must agree exactly
    import ctypes
    import subprocess
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "gwc.h"', "int main(void) {"]
    for py, c in STRUCTS.items():
        cls = getattr(g, py)
        lines.append(f'  printf("{py} size %zu\\n", sizeof({c}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{py} {f} %zu\\n", offsetof({c}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_side = {(a, b): int(n) for a, b, n in (ln.split() for ln in got if ln.strip())}
    for py in STRUCTS:
        cls = getattr(g, py)
        assert c_side[(py, "size")] == ctypes.sizeof(cls), py
        for f, _ in cls._fields_:
            assert c_side[(py, f)] == getattr(cls, f).offset, (py, f)


def test_defaults(g):
    o = g.default_options()
    assert (o.neff_min_event, o.neff_min_sel, o.accum, o.los_dtype) == (2.0, 0.0, 0, 0)
    assert (o.n_x_table, o.max_K, o.chunk, o.lambda_tile, o.lambda_group) == (512, 256, 2048, 0, 0)
    assert (o.cap_per_pixel, o.cap_seed, o.mass_model) == (0, 0, g.MASS_PLP)
    assert g.default_options(mass_model="multipeak").mass_model == g.MASS_MULTIPEAK


def test_invalid_inputs_rejected_before_any_device_work(g, synth):
    import torch
    if torch.cuda.is_available():
        pytest.skip("checks the host-side path on a machine without a GPU")
    w = synth.scaled("t", 3, ("fixed", 50), 2, 16, 100, "draws")
    cat = synth.catalogue(w)
    bad = dict(cat)
    bad["pix"] = cat["pix"].copy()
    bad["pix"][0] = 10_000
    with pytest.raises(g.GwcError) as e:
        g.create(bad)
    assert e.value.status == -1 and "pixel" in str(e.value)
    bad = dict(cat)
    bad["offsets"] = cat["offsets"].copy()
    bad["offsets"][1] = 0
    with pytest.raises(g.GwcError) as e:
        g.create(bad)
    assert e.value.status == -1
    bad = dict(cat)
    bad["dl"] = cat["dl"].copy()
    bad["dl"][3] = np.nan
    with pytest.raises(g.GwcError) as e:
        g.create(bad)
    assert e.value.status == -1
    with pytest.raises(g.GwcError) as e:
        g.create(cat, g.default_options(chunk=8))
    assert e.value.status == -1
    # valid inputs reach the device query, which fails without a GPU
    with pytest.raises(g.GwcError) as e:
        g.create(cat)
    assert e.value.status == -5


def test_null_context_calls_fail_cleanly(g):
    import ctypes
    lib = g.lib()
    assert lib.gwc_loglik(None, 1, None, None, None, None, None, None, None, None) == -1
    assert "context" in g.last_error()
    lib.gwc_destroy(None)
    info = g.Info()
    assert lib.gwc_get_info(None, ctypes.byref(info)) == -1


def test_cap_selection_keeps_the_smallest_keys(g, synth):
    # SplitMix64 reference values (generator started at 1234567): its first outputs
    first = g._splitmix64_outputs(1234567, np.arange(3))
    assert [int(v) for v in first] == [6457827717110365317, 3203168211198807973, 9817491932198370423]
    w = synth.scaled("cap", 6, ("uniform", 300, 900), 8, 128, 1000, "found")
    cat = synth.catalogue(w)
    idx, off = g.cap_selection(cat, 20, seed=99)
    for e in range(6):
        a, b = cat["offsets"][e], cat["offsets"][e + 1]
        sel = idx[off[e]:off[e + 1]]
        assert np.all(np.diff(sel) > 0) and sel.min() >= a and sel.max() < b
        for p in np.unique(cat["pix"][a:b]):
            run = np.arange(a, b)[cat["pix"][a:b] == p]
            kept = sel[cat["pix"][sel] == p]
            assert len(kept) == min(len(run), 20)
            if len(run) > 20:   # exactly the 20 smallest keys of the run
                keys = g._splitmix64_outputs(99, run)
                assert set(kept) == set(run[np.argsort(keys)[:20]])
    other, _ = g.cap_selection(cat, 20, seed=100)
    assert not np.array_equal(idx, other)
    assert len(g.cap_selection(cat, 0)[0]) == len(cat["m1"])
