"""The library used from plain C: a C99 program includes include/cdsdp.h,
links libcdsdp.so and runs the host-only entry points (default options, setup
of the 5-cycle MaxCut relaxation, info, cliques, an invalid input, free).  Its
output must equal what the Python binding reports.  No GPU call."""
import os
import shutil
import subprocess

import pytest

from paper_1707_05058_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r"""
#include <stdio.h>
#include "cdsdp.h"

int main(void) {
    /* MaxCut relaxation of the 5-cycle: C = -L/4 on the cycle, X_ii = 1 */
    int C_row[10], C_col[10];
    double C_val[10];
    int A_con[5], A_row[5], A_col[5];
    double A_val[5], b[5];
    for (int i = 0; i < 5; ++i) {
        C_row[i] = i; C_col[i] = i; C_val[i] = -0.5;
        int j = (i + 1) % 5;
        C_row[5 + i] = i > j ? i : j; C_col[5 + i] = i > j ? j : i; C_val[5 + i] = 0.25;
        A_con[i] = i; A_row[i] = i; A_col[i] = i; A_val[i] = 1.0; b[i] = 1.0;
    }
    cdsdp_opts o;
    cdsdp_default_opts(&o);
    cdsdp* h = NULL;
    int st = cdsdp_setup(5, 5, 5, A_con, A_row, A_col, A_val, b, 10, C_row, C_col, C_val, 0, NULL, NULL, &h);
    if (st != CDSDP_SOLVED) { printf("setup %d\n", st); return 1; }
    cdsdp_info_t info;
    cdsdp_info(h, &info);
    printf("info %d %d %d %d %lld %lld %d\n", info.n, info.m, info.p, info.max_clique, info.nnz_pattern, info.n_fill,
           info.chordal);
    int off[16], vert[64];
    cdsdp_cliques(h, off, vert);
    for (int k = 0; k < info.p; ++k) {
        printf("clique");
        for (int q = off[k]; q < off[k + 1]; ++q) printf(" %d", vert[q]);
        printf("\n");
    }
    cdsdp_free(h);
    /* an upper-triangle entry is rejected */
    int up_row[1] = {0}, up_col[1] = {1};
    double up_val[1] = {1.0};
    cdsdp* h2 = NULL;
    st = cdsdp_setup(5, 5, 5, A_con, A_row, A_col, A_val, b, 1, up_row, up_col, up_val, 0, NULL, NULL, &h2);
    printf("upper %d %s %d\n", st, cdsdp_strerror(st), h2 == NULL);
    printf("eps %g max_iter %d\n", o.eps, o.max_iter);
    return 0;
}
"""


def test_c_client(lib, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(C_SRC)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib.LIB_PATH)
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-lcdsdp", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    P = lib.Problem(W.maxcut_cycle(5))
    inf = P.info
    assert out[0].split() == ["info"] + [str(inf[k]) for k in ("n", "m", "p", "max_clique", "nnz_pattern", "n_fill",
                                                               "chordal")]
    cl = [tuple(int(v) for v in line.split()[1:]) for line in out if line.startswith("clique")]
    assert cl == P.clique_list()
    up = out[-2].split()
    assert up[0] == "upper" and int(up[1]) == -1 and up[-1] == "1"
    assert out[-1] == "eps 0.0001 max_iter 2000"
