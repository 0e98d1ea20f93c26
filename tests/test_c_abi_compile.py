"""include/rsvd.h is a plain C interface: a C99 program compiles against it with
-Wall -Werror, links librsvd.so and runs the host-only calls (option defaults,
status strings, workspace queries, synchronous argument rejection) on CPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "rsvd.h"

int main(void) {
  rsvd_opts o;
  rsvd_opts_default(&o);
  if (o.s != 1 || o.max_sweeps != 30 || o.precision != RSVD_PREC_TC) return 1;
  if (strcmp(rsvd_status_string(RSVD_ERR_WORKSPACE), "RSVD_ERR_WORKSPACE") != 0) return 2;
  if (rsvd_version() < 100) return 3;
  size_t ws = rsvd_svd_id_cur_workspace_size(50000, 20000, 200, 20, 2, RSVD_F32, &o);
  if (ws == 0) return 4;
  if (rsvd_svd_workspace_size(100, 50, 0, 5, 1, RSVD_F32, NULL) != 0) return 5;
  /* invalid arguments are rejected before anything touches a device */
  if (rsvd_qb(100, 50, 10, 5, 1, 7u, RSVD_F32, NULL, 50, NULL, 15, NULL, 15, NULL, 0, NULL,
              NULL, NULL) != RSVD_ERR_INVALID_ARG) return 6;
  int rank = -1;
  double resid[5];
  float buf[4];
  if (rsvd_qb_adaptive(300, 200, 16, 4, 1, -1.0, 1, 7u, RSVD_F32, buf, 200, buf, 64, buf, 64,
                       resid, &rank, NULL, 0, NULL, NULL, NULL) != RSVD_ERR_INVALID_ARG)
    return 7;
  if (rank != -1) return 8;
  printf("ok %zu\n", ws);
  return 0;
}
"""


def test_header_compiles_as_c_and_host_calls_run(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1502_05366_gb300 import build as b
    lib = b.build()
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib)
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           str(src), "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(lib),
           "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ok ")
