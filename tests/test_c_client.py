"""The boundary is a C ABI: include/pastila.h compiles as strict C99, and a plain
C program links against the library and calls its host-only entry points
(argument checks, the runtime model, the device-free layout planner).  CPU
only: nothing here touches a device."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "pastila.h"

int main(void) {
    /* argument errors come back as status codes with a message */
    pastila_series* h = NULL;
    if (pastila_create(&h, NULL, 100, 0, 0, PASTILA_FP32) != PASTILA_EINVAL) return 1;
    if (strstr(pastila_last_error(), "T is NULL") == NULL) return 2;
    /* the runtime model: prior, one observation, a prediction */
    pastila_runtime_model m;
    if (pastila_model_reset(PASTILA_FP32) != PASTILA_OK) return 3;
    if (pastila_model_get(PASTILA_FP32, &m) != PASTILA_OK || m.n_coef != 5 || m.observations != 0) return 4;
    const double f[5] = {1.0, 1.0, 1.0, 0.0, 1.0};
    if (pastila_model_observe(PASTILA_FP32, f, 12.0) != PASTILA_OK) return 5;
    if (pastila_model_get(PASTILA_FP32, &m) != PASTILA_OK || m.observations != 1) return 6;
    const int32_t ms[3] = {64, 128, 256};
    pastila_mparams rule = {0, 0};
    double pred = 0.0;
    if (pastila_model_predict(PASTILA_FP32, 100000, ms, 3, rule, 4, 232448 - 1024, 0.0, &pred) != PASTILA_OK)
        return 7;
    if (!(pred > 0.0)) return 8;
    /* the layout planner without a device */
    int32_t lay[8];
    if (pastila_plan_layout(PASTILA_FP32, 100000, 128, rule, 232448 - 1024, lay) != PASTILA_OK) return 9;
    if (lay[0] % 32 != 0 || lay[2] > 512 || lay[7] > 232448) return 10;
    printf("ok %.3f %d %d\n", pred, lay[0], lay[2]);
    return 0;
}
"""


def test_header_is_strict_c99_and_a_c_program_links(tmp_path):
    from paper_2401_13680_b300 import build
    lib = build.build()
    src = tmp_path / "client.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "client"
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                         "-I", os.path.join(ROOT, "include"), str(src), lib, "-o", str(exe),
                         "-Wl,-rpath," + os.path.dirname(lib)], capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, (run.returncode, run.stdout, run.stderr)
    assert run.stdout.startswith("ok ")
