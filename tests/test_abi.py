"""The C ABI: the library builds, loads, exports every function declared in
include/*.h, and the ctypes structures match the C layout.  No GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2005_12338_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")
HEADERS = sorted(os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h"))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.lib()


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"RSSRI_API\s+[\w\s\*]*?\b(rssri_\w+)\s*\(", text)))


def test_header_declares_the_path():
    names = declared_functions()
    for f in ("rssri_create", "rssri_destroy", "rssri_setup", "rssri_sigma",
              "rssri_sigma_from_g", "rssri_export", "rssri_buffer_bytes", "rssri_status_string"):
        assert f in names
    assert set(names) == set(binding.SIGNATURES)


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (rssri_\w+)", out))
    assert set(declared_functions()) <= exported
    # internal C++ symbols stay hidden
    assert not any("_ZN5rssri" in line for line in out.splitlines())


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "rssri.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(rssri_problem),"
        " sizeof(rssri_options), sizeof(rssri_stats), offsetof(rssri_problem, mu),"
        " offsetof(rssri_options, pair_batch), offsetof(rssri_stats, t_sample_ms));return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                       check=True).stdout.split()))
    want = [C.sizeof(binding.rssri_problem), C.sizeof(binding.rssri_options),
            C.sizeof(binding.rssri_stats), binding.rssri_problem.mu.offset,
            binding.rssri_options.pair_batch.offset, binding.rssri_stats.t_sample_ms.offset]
    assert got == want


def test_status_strings_and_null_handles(lib):
    for code in binding.STATUS:
        assert lib.rssri_status_string(code)
    opts = binding.Handle.options()
    assert lib.rssri_setup(None, None, C.byref(opts)) == -1
    assert lib.rssri_sigma(None, C.byref(opts), None, None, None, None, None) == -1
    assert lib.rssri_export(None, 0, None, 0, 1) == -1
    lib.rssri_destroy(None)
    h = C.c_void_p()
    assert lib.rssri_create(None, 0, None) == -1


def test_no_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    rc = lib.rssri_create(C.byref(h), 0, None)
    assert rc != 0 and not h.value
