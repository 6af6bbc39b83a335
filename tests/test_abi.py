"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/pulda.h declares; the Python binding names the same calls."""
import ctypes
import os
import re

import paper_1704_03581_gb300 as P
from paper_1704_03581_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pulda.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pulda_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    names = declared_symbols()
    assert sorted(P.EXPORTED) == names
    for n in names:
        assert callable(getattr(P, n)), n


def test_init_rejects_bad_arguments_without_a_gpu():
    """Validation happens before any device work, so it is testable on CPU."""
    import numpy as np
    w = np.array([0, 1, 2], np.int32)
    off = np.array([0, 3], np.int64)
    for kwargs, frag in [(dict(K=0), "K must be"), (dict(K=20000), "K must be"), (dict(V=2), "outside"),
                         (dict(alpha=-1.0), "alpha"), (dict(beta=0.0), "beta")]:
        args = dict(K=4, V=3, alpha=0.1, beta=0.01)
        args.update(kwargs)
        try:
            P.pulda_init(w, off, args["K"], args["V"], args["alpha"], args["beta"], 0)
        except P.PuldaError as e:
            assert e.status == -1 and frag in str(e), str(e)
        else:
            raise AssertionError("accepted " + repr(kwargs))
    for kwargs, frag in [(dict(zstep_path=3), "zstep_path"), (dict(warps_per_block=9), "warps_per_block"),
                         (dict(warps_per_block=-1), "warps_per_block"), (dict(docs_per_warp=2), "docs_per_warp"),
                         (dict(phi_mode=2), "phi_mode"), (dict(slice_len=-1), "slice_len"),
                         (dict(slice_len=50, docs_per_warp=4), "slice_len"), (dict(coop_min_len=-2), "coop_min_len"),
                         (dict(count_path=2), "count_path"), (dict(alias_layout=3), "alias_layout"),
                         (dict(alias_layout=-1), "alias_layout")]:
        try:
            P.pulda_init(w, off, 4, 3, 0.1, 0.01, 0, **kwargs)
        except P.PuldaError as e:
            assert e.status == -1 and frag in str(e), str(e)
        else:
            raise AssertionError("accepted " + repr(kwargs))
    bad_off = np.array([0, 2, 1, 3], np.int64)
    try:
        P.pulda_init(w, bad_off, 4, 3, 0.1, 0.01, 0)
    except P.PuldaError as e:
        assert "decrease" in str(e)
    else:
        raise AssertionError("accepted decreasing offsets")


def test_batch_rejects_bad_options_without_a_gpu():
    """The batched form draws the Polya-urn Phi only and caps its CTA at the batched kernel's
    size; both are checked before any device work."""
    import ctypes
    import numpy as np
    w = np.array([0, 1], np.int32)
    off = np.array([0, 2], np.int64)
    a = np.full(3, 0.1, np.float32)
    arr = (P.ChainDesc * 1)()
    arr[0] = P.ChainDesc(P._ptr(w), P._ptr(off), 1, 3, 2, P._ptr(a), 0.01, 0)
    for field, value, frag in [("phi_mode", 1, b"phi_mode"), ("warps_per_block", 9, b"warps_per_block"),
                               ("docs_per_warp", 4, b"docs_per_warp"), ("slice_len", 64, b"slice_len"),
                               ("coop_min_len", -2, b"coop_min_len"), ("count_path", 1, b"count_path"),
                               ("alias_layout", 3, b"alias_layout")]:
        opt = P.Options()
        setattr(opt, field, value)
        b = ctypes.c_void_p()
        st = P.lib().pulda_batch_init(ctypes.byref(b), arr, 1, ctypes.byref(opt))
        assert st == -1 and not b.value
        assert frag in P.lib().pulda_batch_last_error(None), P.lib().pulda_batch_last_error(None)



def test_binding_structures_match_the_header(tmp_path):
    """The ctypes structures of the binding have the C header's sizes and field
    offsets (a C probe compiled against include/pulda.h prints them)."""
    import ctypes
    import os
    import shutil
    import subprocess
    import pytest
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = {"pulda_options": P.Options, "pulda_sweep_stats": P.SweepStats, "pulda_chain_desc": P.ChainDesc,
               "pulda_result": P.ServeResult}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pulda.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ['return 0;', '}']
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run([cc, "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            name, key, val = line.split()
            got[(name, key)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_noalloc_binding_rejects_bad_tensors_before_the_call():
    """pulda_infer_noalloc hands raw device pointers to C, which trusts the
    sizes: the binding refuses wrong dtypes, shapes, strides, a short output
    and host tensors before anything reaches the library (no handle needed)."""
    import pytest
    import torch
    w = torch.zeros(6, dtype=torch.int32)
    off = torch.tensor([0, 2, 6], dtype=torch.int64)
    z = torch.zeros(6, dtype=torch.int16)
    cases = [
        ((w.to(torch.int64), off, z), "word_ids_dev must be int32"),
        ((w, off.to(torch.int32), z), "doc_offsets_dev must be int64"),
        ((w, off, z.to(torch.int32)), "z_out_dev must be int16"),
        ((w.view(2, 3), off, z), "one-dimensional"),
        ((torch.zeros(12, dtype=torch.int32)[::2], off, z), "contiguous"),
        ((w, off, z[:5]), "fewer than the 6 word ids"),
        ((w, torch.zeros(0, dtype=torch.int64), z), "at least one entry"),
        ((w, off, z), "must be a CUDA tensor"),
        (([0, 1], off, z), "must be a torch tensor"),
    ]
    for (a, b, c), frag in cases:
        with pytest.raises(ValueError, match=frag):
            P.pulda_infer_noalloc(None, a, b, 1, 0, c)


def test_allocator_callbacks_must_come_in_pairs():
    """pulda_options' alloc and free are set together or not at all; the
    check comes before any device work (handle and batch)."""
    import ctypes
    import numpy as np
    w = np.array([0, 1, 2], np.int32)
    off = np.array([0, 3], np.int64)
    a = np.full(4, 0.1, np.float32)
    alloc_only = P.ALLOC_FN(lambda n, s, c: None)
    free_only = P.FREE_FN(lambda p, s, c: None)
    for field, fn in (("alloc", alloc_only), ("free", free_only)):
        opt = P.Options()
        setattr(opt, field, fn)
        h = ctypes.c_void_p()
        st = P.lib().pulda_init(ctypes.byref(h), P._ptr(w), P._ptr(off), 1, 4, 3, P._ptr(a), 0.01, 0,
                                ctypes.byref(opt))
        assert st == -1 and not h.value
        assert b"alloc and free" in P.lib().pulda_last_error(None)
        arr = (P.ChainDesc * 1)()
        arr[0] = P.ChainDesc(P._ptr(w), P._ptr(off), 1, 4, 3, P._ptr(a), 0.01, 0)
        b = ctypes.c_void_p()
        st = P.lib().pulda_batch_init(ctypes.byref(b), arr, 1, ctypes.byref(opt))
        assert st == -1 and not b.value
        assert b"alloc and free" in P.lib().pulda_batch_last_error(None)
