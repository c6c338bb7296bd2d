"""The boundary is a C ABI: include/msp.h compiles as plain C (C99, every warning an
error) and a C program that calls every entry point links against libmsp.so.  The
program is compiled and linked here, not run (running it needs a GPU)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "msp.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|long long|const char\*)\s+(msp_\w+)\s*\(",
                                 src, re.M)))


PROGRAM = r"""
#include <stdio.h>
#include "msp.h"

int main(void) {
  msp_config cfg;
  msp_handle h = NULL;
  msp_solve_info info;
  msp_server_config sc;
  msp_request req;
  msp_result res;
  msp_server_stats st;
  msp_server srv = NULL;
  msp_wells w = NULL;
  int64_t t = 0, bytes = 0;
  int32_t g = 0;
  if (msp_config_default(&cfg) != MSP_OK) return 1;
  cfg.precision = MSP_PRECISION_FP32;
  cfg.colouring = MSP_COLOURING_JP;
  cfg.smoother = MSP_SMOOTHER_PGS_MC;
  (void)info; (void)sc; (void)req; (void)res; (void)st; (void)t; (void)bytes; (void)g;
  /* reference every entry point so that the link resolves all of them */
  void *fns[] = {
%s
  };
  printf("%%d entry points, %%s\n", (int)(sizeof fns / sizeof fns[0]), msp_status_string(MSP_OK));
  (void)h; (void)srv; (void)w;
  return 0;
}
"""


def test_header_is_c99_and_links():
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2208_08594_gb300 import _native
    lib = _native.library_path()
    _native.lib()  # builds it if needed
    names = _declared()
    body = "\n".join("    (void *)%s," % n for n in names)
    src = PROGRAM % body
    work = os.path.join(ROOT, "paper_2208_08594_gb300", "_build")
    os.makedirs(work, exist_ok=True)
    c_file = os.path.join(work, "abi_check.c")
    exe = os.path.join(work, "abi_check")
    open(c_file, "w").write(src)
    cuda_lib = "/usr/local/cuda/lib64"
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-Wno-pedantic",
           "-I", os.path.join(ROOT, "include"), c_file, "-o", exe,
           "-L", os.path.dirname(lib), "-l:" + os.path.basename(lib),
           "-Wl,-rpath," + os.path.dirname(lib), "-Wl,--allow-shlib-undefined"]
    if os.path.isdir(cuda_lib):
        cmd += ["-L", cuda_lib, "-Wl,-rpath-link," + cuda_lib]
    out = subprocess.run(cmd, capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    assert os.path.exists(exe)
