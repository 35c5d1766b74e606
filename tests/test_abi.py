"""The C-ABI library builds, loads and exports every symbol include/fg_lattice.h declares.

These run without a GPU: nothing here launches a kernel.
"""

import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

from paper_0910_2950_gb300 import build, fg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(fg_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fg.load()


def test_every_declared_symbol_is_exported(lib):
    names = _header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} declared but not exported"


def test_binding_covers_the_header():
    names = set(_header_functions())
    assert names <= set(fg.SIGNATURES), sorted(names - set(fg.SIGNATURES))


def _header_enums():
    """{enum type name: {enumerator: value}} of the C header's typedef enums."""
    text = open(os.path.join(ROOT, "include", "fg_lattice.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef\s+enum\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
        out[name] = {k: int(v) for k, v in re.findall(r"\b(FG_[A-Z0-9_]+)\s*=\s*(-?\d+)", body)}
    return out


def test_binding_constants_match_the_header_enums():
    """The Python names of statuses, integrators and precisions carry the
    values the C header gives them."""
    enums = _header_enums()
    status = enums["fg_status"]
    for name in ("FG_OK", "FG_EINVAL", "FG_ENOMEM", "FG_ECUDA", "FG_ENOCONV", "FG_ETIMEOUT", "FG_ESTATE"):
        assert getattr(fg, name) == status[name], name
    assert fg.STATUS_NAMES == {v: k for k, v in status.items()}
    prec = enums["fg_precision"]
    assert sorted(fg.PRECISIONS.values()) == sorted(prec.values())
    for key, value in fg.PRECISIONS.items():
        assert prec["FG_" + key.upper()] == value, key
    integ = enums["fg_integrator"]
    assert set(fg.INTEGRATORS.values()) == set(integ.values())
    for key, value in fg.INTEGRATORS.items():
        if "FG_" + key.upper() in integ:
            assert integ["FG_" + key.upper()] == value, key


def test_params_default(lib):
    p = fg.FgParams()
    assert lib.fg_params_default(C.byref(p)) == fg.FG_OK
    assert list(p.dims) == [4, 4, 4, 4]
    assert p.beta == 6.0 and p.kappa == 0.0 and abs(p.alpha - 0.1932) < 1e-15
    assert p.link_reals == 18 and p.cg_tol == 1e-10 and p.cg_maxiter == 20000
    assert lib.fg_params_default(None) == fg.FG_EINVAL


@pytest.mark.parametrize("field,value", [("dims", (3, 4, 4, 4)), ("dims", (4, 4, 0, 4)),
                                         ("dims", (130, 128, 128, 128)),   # over 2^28 sites
                                         ("link_reals", 10), ("precision", 6), ("precision", -1),
                                         ("cg_maxiter", 0),
                                         ("cg_tol", 0.0), ("cg_delta", 1.5)])
def test_create_rejects_bad_parameters_before_touching_the_device(lib, field, value):
    p = fg.FgParams()
    lib.fg_params_default(C.byref(p))
    if field == "dims":
        for i, d in enumerate(value):
            p.dims[i] = d
    else:
        setattr(p, field, value)
    h = C.c_void_p()
    assert lib.fg_lattice_create(C.byref(p), C.byref(h)) == fg.FG_EINVAL
    assert not h.value


def test_double_float_handles_are_pure_gauge(lib):
    p = fg.FgParams()
    lib.fg_params_default(C.byref(p))
    p.precision = fg.PRECISIONS["df64"]
    p.kappa = 0.158
    h = C.c_void_p()
    assert lib.fg_lattice_create(C.byref(p), C.byref(h)) == fg.FG_EINVAL
    assert not h.value


def test_noalloc_rejects_oversized_extents_before_touching_the_device(lib):
    # the site count is checked after every factor, so huge extents cannot
    # overflow the product into an accepted size
    for dims in ([1 << 30] * 4, [2, 2, 1 << 30, 1 << 30], [1 << 24, 2, 2, 2], [4096, 4096, 2, 2]):
        d = (C.c_int * 4)(*dims)
        assert lib.fg_action_sums_noalloc(C.c_void_p(256), None, d, 6.0, C.c_void_p(256), None) == fg.FG_EINVAL


def test_wait_limit_validation(lib):
    assert lib.fg_set_wait_limit(None, 1.0) == fg.FG_EINVAL
    assert lib.fg_batch_set_wait_limit(None, 1.0) == fg.FG_EINVAL


def test_bounded_host_wait_logic(tmp_path):
    """The polling loop behind fg_set_wait_limit (csrc/host_wait.h), built as
    plain C++ and driven by a fake clock: work that never finishes times out
    once the limit has passed, work that finishes or fails is reported as
    such, and the pause between polls grows to 1 ms."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "wait.cpp"
    src.write_text(r'''
#include <cstdio>
#include "host_wait.h"
int main() {
  using namespace fg;
  double t = 0.0, slept = 0.0, last = 0.0;
  int polls = 0;
  auto now = [&] { return t; };
  auto pause = [&](double us) { t += us * 1e-6; slept += us; last = us; };
  // never finishes: times out after the limit
  WaitResult w = wait_limited([&] { ++polls; return 1; }, now, pause, 0.05);
  if (w != WAIT_TIMEOUT || t < 0.05 || t > 0.052 || last != 1000.0) { std::printf("timeout %d %g %g\n", w, t, last); return 1; }
  // finishes at the fourth poll
  t = 0.0; polls = 0;
  w = wait_limited([&] { return ++polls >= 4 ? 0 : 1; }, now, pause, 0.05);
  if (w != WAIT_DONE || polls != 4) { std::printf("done %d %d\n", w, polls); return 1; }
  // an error is reported at once
  t = 0.0; polls = 0;
  w = wait_limited([&] { ++polls; return 7; }, now, pause, 0.05);
  if (w != WAIT_ERROR || polls != 1) { std::printf("error %d %d\n", w, polls); return 1; }
  std::printf("ok\n");
  return 0;
}
''')
    exe = tmp_path / "wait"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.join(root, "paper_0910_2950_gb300", "csrc"), str(src),
                    "-o", str(exe)], check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert res.returncode == 0 and res.stdout.strip() == "ok", res.stdout


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.fg_refresh_momenta(None) == fg.FG_EINVAL
    assert lib.fg_sync(None) == fg.FG_EINVAL
    assert lib.fg_launch_count(None) == -1
    assert lib.fg_last_error(None) == b"null handle"
    lib.fg_lattice_destroy(None)
    assert lib.fg_trajectories_host_momenta(None, 2, 0.25, 1.0, 0, None, None, None) == fg.FG_EINVAL
    assert lib.fg_trajectories_host_momenta_f32(None, 2, 0.25, 1.0, 0, None, None, None) == fg.FG_EINVAL
    assert lib.fg_fp32_fma_rate(None) == fg.FG_EINVAL


@pytest.mark.parametrize("case", ["odd", "too_large", "tile", "link_reals", "df64_tile64", "df64_12real"])
def test_batch_create_rejects_bad_parameters_before_touching_the_device(lib, case):
    dims = [4, 4, 4, 4, 6, 6, 6, 6]
    if case == "odd":
        dims[5] = 5
    elif case == "too_large":
        dims[4:] = [130, 128, 128, 128]
    betas = [6.0, 5.8]
    p = fg.FgBatchParams()
    lib.fg_batch_params_default(C.byref(p))
    p.nchains = 2
    d = (C.c_int * 8)(*dims)
    b = (C.c_double * 2)(*betas)
    p.dims = C.cast(d, C.POINTER(C.c_int))
    p.beta = C.cast(b, C.POINTER(C.c_double))
    if case == "tile":
        p.tile = 48
    elif case == "link_reals":
        p.link_reals = 16
    elif case == "df64_tile64":       # double-float batches compile tiles of 16 and 32 half-sites only
        p.precision, p.tile = fg.PRECISIONS["df64"], 64
    elif case == "df64_12real":       # and 18-real links only
        p.precision, p.link_reals = fg.PRECISIONS["df64"], 12
    h = C.c_void_p()
    assert lib.fg_batch_create(C.byref(p), C.byref(h)) == fg.FG_EINVAL
    assert not h.value


def _cc():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    return cc


def test_header_and_example_build_as_plain_c(lib, tmp_path):
    """The ABI is usable from strict C99: the header alone, and the example
    chain program compiled and linked against the library (not run: no GPU)."""
    cc = _cc()
    inc = os.path.join(ROOT, "include")
    pkg = os.path.join(ROOT, "paper_0910_2950_gb300")
    flags = ["-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc]
    hdr_only = tmp_path / "h.c"
    hdr_only.write_text('#include "fg_lattice.h"\nint main(void) { return FG_OK; }\n')
    subprocess.run([cc] + flags + ["-c", str(hdr_only), "-o", str(tmp_path / "h.o")], check=True)
    exe = tmp_path / "hmc_chain"
    subprocess.run([cc] + flags + [os.path.join(pkg, "examples", "hmc_chain.c"), "-L", pkg, "-l:libfg_lattice.so",
                                   "-Wl,-rpath," + pkg, "-lm", "-o", str(exe)], check=True)
    assert exe.exists()
