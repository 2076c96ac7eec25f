"""The launch-time iteration limit that keeps the grid barrier's 32-bit arrival count from
wrapping (check_barrier_budget, a host function): compiled with nvcc into a small host
program linked against the library and run without a GPU.  It must accept every solve the
benchmarks and tests run and refuse the first max_it past the limit it reports."""
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SOURCE = r"""
#include <cstdio>
#include <cstring>
#include "capi_internal.h"

static int ok(int max_it, int restarts, int degree, int blocks, int restart_period = 0, int stag = 0) {
  return check_barrier_budget(max_it, restarts, degree, blocks, restart_period, stag) == PBCG_OK;
}

int main() {
  // configurations the benchmarks and tests run: 2D (152 blocks), 3D streaming Neumann-2
  // (456 blocks), the 16-RHS teams (19 blocks), launch-shape sweeps (up to 1216 blocks)
  if (!ok(20000, 0, 0, 152) || !ok(20000, 0, 2, 456) || !ok(30000, 3, 0, 19) || !ok(20000, 3, 0, 1216)) return 1;
  if (!ok(0, 0, 8, 4096)) return 2;
  // far past the limit
  if (ok(2000000, 0, 0, 152) || ok(400000, 0, 2, 456)) return 3;
  // the limit the message reports is accepted, the next value refused
  const int cases[][3] = {{0, 0, 152}, {2, 0, 456}, {0, 3, 19}, {8, 1000, 1}};
  for (const auto& c : cases) {
    if (check_barrier_budget(2147483647, c[1], c[0], c[2]) != PBCG_INVALID_ARG) return 4;
    const char* msg = pbicgstab_last_error();
    const char* at = strstr(msg, "at most ");
    if (!at) return 5;
    long long lim = 0;
    if (sscanf(at + 8, "%lld", &lim) != 1 || lim < 1) return 6;
    if (!ok((int)lim, c[1], c[0], c[2]) || ok((int)lim + 1, c[1], c[0], c[2])) return 7;
  }
  // with a restart policy (restart every 75 iterations, stagnation window): the benchmark's
  // mixed 2D solve (304 blocks of the four-row kernel) and 3D solves are accepted
  if (!ok(20000, 0, 0, 304, 75, 4000) || !ok(20000, 0, 2, 152, 100, 4000)) return 8;
  // a restart policy costs up to one (re)start per iteration, so its limit is lower
  {
    if (check_barrier_budget(2147483647, 0, 2, 152, 100, 1) != PBCG_INVALID_ARG) return 9;
    const char* at = strstr(pbicgstab_last_error(), "at most ");
    long long lim = 0;
    if (!at || sscanf(at + 8, "%lld", &lim) != 1 || lim < 1) return 10;
    if (!ok((int)lim, 0, 2, 152, 100, 1) || ok((int)lim + 1, 0, 2, 152, 100, 1)) return 11;
    if (!ok((int)lim + 1, 0, 2, 152, 0, 0)) return 12;   // without restarts the same max_it fits
  }
  printf("ok\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def libdir():
    from paper_1809_01948_gb300._build import build, _nvcc
    return os.path.dirname(build()), _nvcc()


def test_barrier_budget_limits(libdir):
    lib, nvcc = libdir
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "budget.cu"), os.path.join(d, "budget")
        open(src, "w").write(SOURCE)
        subprocess.check_call([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                               "-I", os.path.join(ROOT, "paper_1809_01948_gb300", "csrc"),
                               "-I", os.path.join(ROOT, "include"), src, "-L", lib, "-lpbicgstab",
                               "-Xlinker", "-rpath=" + lib, "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
