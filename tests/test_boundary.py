"""The C ABI boundary without a GPU: the library loads, exports every entry
point include/rt.h declares, and rejects bad arguments on the host."""
import re
import os

import numpy as np
import pytest

from paper_2208_05247_b300 import build, rt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b((?:rt|nn)_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return rt.library()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert "rt_trace" in names and "rt_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2208_05247_b300 import nn
    for n in _declared():
        mod = nn if n.startswith("nn_") else rt
        assert callable(getattr(mod, n)), n


def test_create_rejects_bad_sizes(lib):
    for args in [(0, 4, 4, 1, 1, 1), (4, -1, 4, 1, 1, 1), (4, 4, 4, 0.0, 1, 1), (4, 4, 4, 1, float("nan"), 1),
                 (2048, 2048, 1024, 1, 1, 1)]:
        with pytest.raises(rt.RtError) as e:
            rt.rt_create(*args)
        assert e.value.code == rt.RT_E_INVAL


def test_debug_entry_points_reject_bad_arguments(lib):
    with pytest.raises(rt.RtError):
        rt.rt_debug_sample("hg", 10, g=1.0)
    with pytest.raises(ValueError):
        rt.rt_debug_philox(np.zeros((2, 4)), np.zeros((3, 2)))


def test_binding_checks_buffers_before_calling():
    with pytest.raises(ValueError):
        rt.rt_set_optics(None, 8, *[np.zeros(8, np.float64)] * 5)
    with pytest.raises(ValueError):
        rt.rt_set_optics(None, 8, *[np.zeros(7, np.float32)] * 5)
    with pytest.raises(ValueError):
        rt.rt_fields(None, 8, 4, abs3d=np.zeros(8, np.float32))
    with pytest.raises(TypeError):
        rt.rt_set_surface(None, 4, [0.1, 0.2, 0.3, 0.4])


def test_null_handle_is_an_error(lib):
    with pytest.raises(rt.RtError) as e:
        rt.rt_build_accel(None)
    assert e.value.code == rt.RT_E_INVAL


def test_no_gpu_means_a_loud_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rt.RtError) as e:
        rt.rt_create(4, 4, 4, 1, 1, 1)
    assert e.value.code in (rt.RT_E_CUDA, rt.RT_E_OOM)


C_CALLER = r"""
#include <stdio.h>
#include <string.h>
#include "rt.h"
#include "nn.h"

/* A plain C caller: without a usable GPU rt_create returns NULL and leaves a
   message; argument checks fail before any device work. */
int main(void)
{
    rt_handle h = rt_create(32, 32, 32, 100.0, 100.0, 100.0);
    if (h) {
        rt_destroy(h);
        printf("handle\n");
        return 0;
    }
    printf("code %d: %s\n", rt_last_error_code(), rt_last_error());
    return strlen(rt_last_error()) > 0 ? 0 : 1;
}
"""


def test_headers_are_c99_and_a_c_program_links(lib, tmp_path):
    """include/*.h compile as C99 (no C++ in the ABI), and a C program links
    against the library and gets a loud error, not a crash, without a GPU."""
    import subprocess
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(rt.LIB)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           str(src), "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(rt.LIB), "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.stdout, r.stderr)
    import torch
    if not torch.cuda.is_available():
        assert r.stdout.startswith("code "), r.stdout


def test_readme_c_example_compiles(tmp_path):
    """The C usage example in README.md compiles against include/rt.h."""
    import subprocess
    text = open(os.path.join(ROOT, "README.md")).read()
    block = re.search(r"```c\n(.*?)```", text, flags=re.S).group(1)
    body = "\n".join(ln for ln in block.splitlines() if not ln.startswith("#include"))
    src = tmp_path / "example.c"
    src.write_text('#include <stdint.h>\n#include "rt.h"\n'
                   "void example(int nx, int ny, int nz, const float *k_gas, const float *ssa_gas,\n"
                   "             const float *k_cld, const float *ssa_cld, const float *g_cld, const float *albedo,\n"
                   "             double *abs3d, double *sfc_dir, double *sfc_dif, double *toa_up)\n{\n"
                   + body + "\n}\n")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
