"""The C ABI from a plain C program (no Python, no GPU): a C99 client built
with gcc against include/diffsoup.h and the library calls the host-only
entry points -- the version, the adaptive-control plans, an argument check
and the error message."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r"""
#include <stdio.h>
#include <string.h>
#include "diffsoup.h"

int main(void) {
    int32_t counts[3] = {3, 0, 7};
    float ratios[9] = {0.3f, 0.1f, 0.0f, 0.0f, 0.0f, 0.0f, 0.1f, 0.25f, 0.26f};
    int32_t plan[6], n = -1;
    if (ds_version() <= 0) return 1;
    if (ds_adapt_plan(counts, ratios, 3, 0.2f, -1, plan, &n) != DS_OK || n != 5) return 2;
    if (plan[0] != (0 << 3 | 1) || plan[2] != (1 << 3) || plan[3] != (2 << 3 | 5)) return 3;
    if (ds_adapt_plan_fill(counts, ratios, 3, 3, plan, &n) != DS_OK || n != 3) return 4;
    if (ds_adam_step(NULL, NULL, NULL, NULL, 12, 5, 0.1f, 0.9f, 0.999f, 1e-8f, 1, NULL) != DS_ERR_INVALID_ARG) return 5;
    if (strlen(ds_last_error()) == 0) return 6;
    printf("ok %d\n", (int)n);
    return 0;
}
"""


def test_c_client(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    import __graft_entry__
    __graft_entry__.build()
    lib_dir = os.path.join(ROOT, "paper_2603_27151_gb300", "_lib")
    src = tmp_path / "client.c"
    src.write_text(SRC)
    exe = tmp_path / "client"
    subprocess.check_call([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe), "-L", lib_dir, "-ldiffsoup", "-Wl,-rpath," + lib_dir])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok 3", (r.returncode, r.stdout, r.stderr)
