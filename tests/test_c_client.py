"""The boundary is a C ABI: a plain C99 program includes include/fdk.h,
links libfdk.so and calls it.  No GPU is needed: the calls made here either
need no device (version, error text, a zero-view no-op) or fail in the
argument checks, which run before any CUDA call."""
import os
import shutil
import subprocess

import pytest

from paper_1401_3615_gb300 import build as fdk_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "fdk.h"

int main(void)
{
    const int32_t dims[3] = {4, 4, 4}, det[2] = {8, 8}, bad_dims[3] = {4, 0, 4};
    const float vs[3] = {1.0f, 1.0f, 1.0f}, org[3] = {0.0f, 0.0f, 0.0f};
    float mats[12];
    fdk_opts opts;
    fdk_status st;
    int q;
    for (q = 0; q < 12; ++q) mats[q] = 1.0f;
    memset(&opts, 0, sizeof opts);
    if (fdk_version() != 1) return 10;
    /* zero views: a no-op that needs no device */
    st = fdk_backproject((float *)0x100, dims, vs, org, NULL, det, mats, 0, &opts);
    if (st != FDK_OK || strcmp(fdk_last_error(), "") != 0) return 11;
    /* a bad size is refused before any CUDA call, with a message */
    st = fdk_backproject((float *)0x100, bad_dims, vs, org, (const void *)0x100, det, mats, 1, NULL);
    if (st != FDK_ERR_INVALID_ARG || strstr(fdk_last_error(), "dims") == NULL) return 12;
    /* an unknown option likewise */
    opts.fetch = 9;
    st = fdk_forwardproject_adjoint((void *)0x100, det, (const float *)0x100, dims, vs, org, mats, 1, &opts);
    if (st != FDK_ERR_INVALID_ARG) return 13;
    printf("ok %d\n", (int)sizeof(fdk_opts));
    return 0;
}
"""


def test_c99_client_compiles_links_and_calls(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = fdk_build.build()
    src = tmp_path / "client.c"
    src.write_text(CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                        "-L", libdir, "-lfdk", f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ok ")
