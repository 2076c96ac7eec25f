"""A plain C program compiles against include/pbicgstab.h, links libpbicgstab.so and drives
the host side of the ABI without a GPU: default options, and the documented INVALID_ARG
paths of create, batch create and the propagation diagnostics, with their messages."""
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SOURCE = r"""
#include <stdio.h>
#include <string.h>
#include "pbicgstab.h"

int main(void) {
  pbcg_options o;
  if (pbicgstab_default_options(&o) != PBCG_OK) return 10;
  if (o.precision != PBCG_FP64 || o.max_it <= 0 || !(o.tol > 0.0) || o.rr_period != 0) return 11;
  pbcg_matrix A;
  memset(&A, 0, sizeof A);
  A.format = PBCG_FMT_CSR;
  A.val_dtype = PBCG_F64;
  A.n = 0;                                   /* empty system: rejected before any CUDA call */
  pbcg_precond M = {PBCG_PREC_JACOBI, 0};
  pbcg_ctx* ctx = (pbcg_ctx*)0x1;
  if (pbicgstab_create(&ctx, &A, &M, &o, NULL) != PBCG_INVALID_ARG || ctx != NULL) return 12;
  if (strlen(pbicgstab_last_error()) == 0) return 13;
  if (pbicgstab_create(NULL, &A, &M, &o, NULL) != PBCG_INVALID_ARG) return 14;
  pbcg_batch B;
  memset(&B, 0, sizeof B);
  pbcg_batch_ctx* bctx = NULL;
  if (pbicgstab_batch_create(&bctx, &B, &o, NULL) != PBCG_INVALID_ARG) return 15;
  if (pbicgstab_propagation_norms(NULL, 8, 3, NULL, NULL) != PBCG_INVALID_ARG) return 16;
  if (pbicgstab_destroy(NULL) != PBCG_OK || pbicgstab_batch_destroy(NULL) != PBCG_OK) return 17;
  printf("ok %s\n", pbicgstab_last_error());
  return 0;
}
"""


@pytest.fixture(scope="module")
def libdir():
    from paper_1809_01948_gb300._build import build
    return os.path.dirname(build())


def test_c_program_links_and_validates(libdir):
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "client.c"), os.path.join(d, "client")
        open(src, "w").write(C_SOURCE)
        subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), src,
                               "-L", libdir, "-lpbicgstab", "-Wl,-rpath," + libdir, "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert out.stdout.startswith("ok ")
