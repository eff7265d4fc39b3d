"""The C-ABI library builds, loads and exports every entry point of include/nb.h.

CPU only: no compute call is made without a GPU.
"""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_cs_0702135_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["nb_init", "nb_predict", "nb_force", "nb_correct", "nb_step", "nb_energy",
                     "nb_get_state", "nb_set_state", "nb_free", "nb_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(nb_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_symbol_and_loads(built):
    import ctypes
    import paper_cs_0702135_gb300 as nb
    L = nb.lib()
    bound = {name for name, _, _ in nb.nb.SIGNATURES}
    assert set(_declared()) <= bound
    for name in _declared():
        assert isinstance(getattr(L, name), ctypes._CFuncPtr)


def test_default_opts_without_gpu(built):
    import paper_cs_0702135_gb300 as nb
    o = nb.nb_default_opts()
    assert (o.eta, o.eta_init, o.level_min, o.level_fixed, o.precision) == (0.01, 0.01, 3, 0, nb.NB_DS)
    assert nb.nb_num_particles(None) == -1
    assert nb.nb_last_error(None)


def test_init_rejects_bad_arguments_before_touching_a_device(built):
    # Argument checks run before any CUDA call, so they work on a CPU-only host.
    import numpy as np
    import paper_cs_0702135_gb300 as nb
    m = np.ones(4) / 4
    x = np.random.default_rng(0).normal(size=(4, 3))
    v = np.zeros((4, 3))
    bad = [
        dict(eps=-1.0),
        dict(eps=float("nan")),
        dict(m=np.array([0.5, -0.5, 0.5, 0.5])),
        dict(x=np.where(np.arange(12).reshape(4, 3) == 5, np.inf, x)),
        dict(opts=nb.nb_default_opts(eta=0.0)),
        dict(opts=nb.nb_default_opts(level_min=41)),
        dict(opts=nb.nb_default_opts(level_fixed=2)),
        dict(opts=nb.nb_default_opts(precision=7)),
        dict(opts=nb.nb_default_opts(force_mode=9)),
        dict(opts=nb.nb_default_opts(summation=4)),
        dict(opts=nb.nb_default_opts(summation=nb.NB_SUM_FIXED, precision=nb.NB_FP64)),
        dict(opts=nb.nb_default_opts(summation=nb.NB_SUM_FIXED), eps=0.0),
        dict(opts=nb.nb_default_opts(summation=nb.NB_SUM_FIXED), eps=1e-30),
    ]
    for case in bad:
        args = dict(m=m, x=x, v=v, eps=0.1, opts=None)
        args.update(case)
        with pytest.raises(nb.NbError) as ei:
            nb.nb_init(args["m"], args["x"], args["v"], args["eps"], args["opts"])
        assert ei.value.code == nb.NB_EINVAL, case


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_cs_0702135_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower(), f


def test_binding_structs_match_the_header(tmp_path):
    # offsets and sizes of nb_opts and nb_stats as the C compiler lays them out
    import ctypes
    import paper_cs_0702135_gb300 as nb
    prog = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "nb.h"', 'int main(void) {']
    for st in (nb.nb.nb_opts, nb.nb.nb_stats):
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (st.__name__, st.__name__))
        for name, _ in st._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (st.__name__, name, st.__name__, name))
    lines += ['return 0;', '}']
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(prog)], check=True)
    c_layout = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                             check=True).stdout.splitlines())
    for st in (nb.nb.nb_opts, nb.nb.nb_stats):
        assert int(c_layout[st.__name__]) == ctypes.sizeof(st)
        for name, _ in st._fields_:
            assert int(c_layout["%s.%s" % (st.__name__, name)]) == getattr(st, name).offset, name


def test_default_opts_rejects_unknown_fields(built):
    import paper_cs_0702135_gb300 as nb
    with pytest.raises(TypeError):
        nb.nb_default_opts(sumation=1)


def test_device_wrappers_check_tensors_before_the_call():
    # The device-pointer wrappers refuse tensors of the wrong dtype, on the
    # host, non-contiguous or too short before anything reaches the library
    # (a float32 position array would otherwise be read past its end, an
    # int64 index array as pairs of int32).
    torch = pytest.importorskip("torch")
    import paper_cs_0702135_gb300 as nb
    n = 10
    raw = 1 << 20               # an int is a raw device address: not inspected
    x = torch.zeros((n, 3), dtype=torch.float64)
    idx = torch.zeros(3, dtype=torch.int32)
    cases = [(raw, x.float(), raw, "d_x must be a float64"),
             (raw, raw, idx.long(), "d_active_idx must be a int32"),
             (raw, x, raw, "d_x must be a CUDA"),
             (raw, raw, idx, "d_active_idx must be a CUDA")]
    for dm, dx, di, what in cases:
        with pytest.raises(ValueError, match=what):
            nb.nb_force_few_noalloc(n, dm, dx, raw, 0.1, di, 3, raw)
    with pytest.raises(ValueError, match="d_active_idx must be a int32"):
        nb.nb_force_dev(None, idx.long(), 3, raw)
    assert nb.nb._dev(raw, "float64", 3, "d_x").value == raw
    with pytest.raises(ValueError, match="required"):
        nb.nb._dev(None, "float64", 3, "d_x")
