"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(bo_\w+)\s*\(", text):
            if not m.group(1).endswith("_fn"):
                names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def library():
    from paper_2111_14991_gb300 import build
    build.build()
    from paper_2111_14991_gb300 import bo
    return bo.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for core in ("bo_space_create", "bo_observe", "bo_suggest", "bo_space_destroy",
                 "bo_last_error", "bo_predict"):
        assert core in names


def test_every_declared_symbol_is_exported(library):
    missing = [n for n in sorted(declared_symbols()) if not hasattr(library, n)]
    assert not missing, missing


def test_binding_covers_the_header(library):
    from paper_2111_14991_gb300 import bo
    assert declared_symbols() <= set(bo.SIGNATURES)


def test_struct_layouts_match_header():
    """ctypes mirrors of the C structs have the sizes the C compiler gives them."""
    import ctypes
    import subprocess
    import tempfile
    from paper_2111_14991_gb300 import bo
    src = r'''
#include <stdio.h>
#include "bo_suggest.h"
int main(void) { printf("%zu %zu %zu\n", sizeof(bo_space_desc), sizeof(bo_suggest_info),
                        sizeof(bo_pass_result)); return 0; }
'''
    with tempfile.TemporaryDirectory() as tmp:
        c = os.path.join(tmp, "s.c")
        exe = os.path.join(tmp, "s")
        open(c, "w").write(src)
        subprocess.run(["gcc", c, "-I", os.path.join(ROOT, "include"), "-o", exe], check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True,
                                                check=True).stdout.split()]
    assert sizes == [ctypes.sizeof(bo.SpaceDesc), ctypes.sizeof(bo.SuggestInfo),
                     ctypes.sizeof(bo.PassResult)]


def test_no_gpu_means_loud_failure():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2111_14991_gb300 import Space
    with pytest.raises(RuntimeError):
        Space([[0.0, 1.0]])


def test_noalloc_argument_checks_without_device(library):
    """bo_acquire_noalloc rejects an oversized count and an unknown explore mode
    before it touches any device (so this runs on a machine without a GPU)."""
    from paper_2111_14991_gb300 import bo
    p = bo.AcqParams()
    p.n_cand, p.n_unvisited, p.n_af = 4194304 + 1, 10, 1
    with pytest.raises(bo.BOError) as e:
        bo.acquire_noalloc(16, 16, 16, 0, p, 16, 0)
    assert e.value.code == 11
    p.n_cand, p.explore = 100, 7
    with pytest.raises(bo.BOError) as e:
        bo.acquire_noalloc(16, 16, 16, 0, p, 16, 0)
    assert e.value.code == 1 and "explore" in str(e.value)
