"""The C ABI on a machine without a GPU: the library builds, loads, and exports every
function include/pget.h declares; the Python binding binds exactly those; structure
layouts agree between the header and the binding.  No compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pget.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pget_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_26745_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("pget_forward", "pget_jvp", "pget_vjp", "pget_lm_solve", "pget_cg_solve",
                 "pget_reg_apply", "pget_create", "pget_destroy", "pget_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    L, path = lib
    for name in _declared():
        assert hasattr(L, name), name


def test_binding_matches_header(lib):
    from paper_2604_26745_gb300 import pget
    assert sorted(pget.exported_symbols()) == _declared()


def test_struct_sizes_match_header(lib):
    """Compile a tiny C program against the header and compare sizeof with ctypes."""
    import subprocess
    import tempfile
    from paper_2604_26745_gb300 import pget
    prog = r'''
#include <stdio.h>
#include "pget.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(pget_geometry), sizeof(pget_lm_params),
         sizeof(pget_lm_report), sizeof(pget_kernel_stat), sizeof(pget_trial_report),
         sizeof(pget_check_report));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    assert sizes == [ctypes.sizeof(pget.pget_geometry), ctypes.sizeof(pget.pget_lm_params),
                     ctypes.sizeof(pget.pget_lm_report), ctypes.sizeof(pget.pget_kernel_stat),
                     ctypes.sizeof(pget.pget_trial_report), ctypes.sizeof(pget.pget_check_report)]


def test_no_gpu_calls_fail_cleanly(lib):
    """Without a device, creating a context returns an error status, never aborts."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2604_26745_gb300 import pget
    with pytest.raises(pget.PgetError):
        pget.Context(0)
    assert pget.pget_version().startswith("pget-gb300")


def test_geometry_info_and_depth_table_checks(lib, O):
    """pget_geometry_info is host-only: it reports the samples per ray T of the oracle's
    geometry (the length of the depth tables of Eq. (5)) and rejects invalid tables."""
    import numpy as np
    from paper_2604_26745_gb300 import pget
    for args in ((128, 360, 182, 5), (27, 17, 91, 3), (64, 90, 91, 1)):
        info = pget.geometry_info(pget.geometry(*args[:3], n_sub=args[3]))
        assert info["n_samples"] == O.geom_info(O.geom(*args[:3], n_sub=args[3]))["T"]
    T = pget.geometry_info(pget.geometry(16, 8, 91))["n_samples"]
    ok = pget.geometry(16, 8, 91, depth_w=np.ones(T), depth_c=np.full(T, 1.5))
    assert pget.geometry_info(ok)["n_samples"] == T
    for bad in (dict(depth_w=-np.ones(T)), dict(depth_c=np.full(T, np.nan)), dict(depth_c=np.full(T, np.inf))):
        with pytest.raises(ValueError):
            pget.geometry_info(pget.geometry(16, 8, 91, **bad))
    with pytest.raises(ValueError):  # wrong length
        pget.geometry(16, 8, 91, depth_w=np.ones(T + 1))


def test_plain_c_program_links_and_runs(lib, O):
    """A C program linked against libpget.so (no Python) uses the host-only calls:
    pget_geometry_info gives the oracle's derived sizes, an invalid geometry returns
    PGET_EINVAL, pget_default_params fills the documented defaults, a compute call with null
    arrays returns PGET_EINVAL (through its NVTX range), and without a GPU pget_create
    returns an error status with a message and leaves *ctx NULL."""
    import subprocess
    import tempfile
    import torch
    L, path = lib
    prog = r'''
#include <stdio.h>
#include <string.h>
#include "pget.h"
int main(void) {
  pget_geometry g;
  memset(&g, 0, sizeof g);
  g.n = 128; g.n_angles = 360; g.n_det = 182; g.n_sub = 5; g.collimator = 1;
  int32_t T = 0, nb = 0, slots = 0;
  double r = 0, p = 0;
  int s = pget_geometry_info(&g, &T, &nb, &r, &p, &slots);
  pget_geometry bad = g;
  bad.n = 1;
  int sbad = pget_geometry_info(&bad, NULL, NULL, NULL, NULL, NULL);
  pget_lm_params prm;
  pget_default_params(&prm);
  pget_ctx* ctx = (pget_ctx*)&g;
  int sc = pget_create(&ctx, 0, 0);
  const char* msg = pget_last_error(NULL);
  int snull = pget_forward(NULL, &g, PGET_F32, NULL, NULL, NULL, NULL);  /* opens and closes a range */
  printf("%d %d %d %.17g %.17g %d %d %.17g %.17g %d %d %d %d\n", s, T, nb, r, p, slots, sbad,
         prm.lambda_max, prm.mu_max, sc, ctx == NULL, msg && msg[0] != 0, snull);
  if (sc == PGET_OK) pget_destroy(ctx);
  printf("%s\n", pget_version());
  return 0;
}'''
    d = os.path.dirname(path)
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "use.c")
        open(c, "w").write(prog)
        exe = os.path.join(td, "use")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe, "-L", d, "-lpget",
                        f"-Wl,-rpath,{d}"], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120, check=True).stdout.split("\n")
    f = out[0].split()
    info = O.geom_info(O.geom(128, 360, 182, n_sub=5))
    assert int(f[0]) == 0 and int(f[1]) == info["T"] and int(f[2]) == info["n_banks"] == 2
    assert abs(float(f[3]) - info["radius"]) <= 1e-12 and abs(float(f[4]) - info["pitch"]) <= 1e-12
    assert 91 <= int(f[5]) <= 1024  # distinct rays per view of one bank
    assert int(f[6]) == 1  # PGET_EINVAL
    assert float(f[7]) == 2.0 and float(f[8]) == 0.2
    if not torch.cuda.is_available():
        assert int(f[9]) != 0 and int(f[10]) == 1 and int(f[11]) == 1
    assert int(f[12]) == 1  # PGET_EINVAL for null arrays, through the profiler range
    assert out[1].startswith("pget-gb300")


def test_status_codes_match_header(lib):
    """The binding's status constants are the header's enum, value for value."""
    from paper_2604_26745_gb300 import pget
    src = open(HEADER).read()
    body = src[src.index("typedef enum {"):src.index("} pget_status;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    codes = dict((k, int(v)) for k, v in re.findall(r"(PGET_[A-Z]+)\s*=\s*(\d+)", body))
    assert len(codes) == 9 and sorted(codes.values()) == list(range(9))
    for k, v in codes.items():
        assert getattr(pget, k) == v, k


def test_geometry_limits(lib):
    """Sizes outside the documented ranges are rejected on the host, never computed."""
    from paper_2604_26745_gb300 import pget
    assert pget.geometry_info(pget.geometry(16, 4096, 91))["n_banks"] == 1
    for bad in (dict(n=16, n_angles=(1 << 20) + 1, n_det=91), dict(n=16, n_angles=0, n_det=91),
                dict(n=16385, n_angles=8, n_det=91), dict(n=1, n_angles=8, n_det=91),
                dict(n=16, n_angles=8, n_det=91, n_sub=65)):
        kw = dict(bad)
        with pytest.raises(ValueError):
            pget.geometry_info(pget.geometry(kw.pop("n"), kw.pop("n_angles"), kw.pop("n_det"), **kw))
    import time
    t0 = time.perf_counter()
    with pytest.raises(ValueError, match="detectors per bank"):  # refused before any table is sized
        pget.geometry_info(pget.geometry(16, 8, 2 ** 31 - 1, n_sub=64))
    with pytest.raises(pget.PgetError) as e:  # 2^21 views x 275 rays: tables refused, not built
        pget.geometry_info(pget.geometry(64, 1 << 20, 182, n_sub=5))
    assert e.value.status == pget.PGET_ENOMEM
    assert time.perf_counter() - t0 < 5.0
