"""Memory safety of the oracle's C code, checked with AddressSanitizer on the host CPU.

The oracle's per-target least-squares solve (Sec. 3.2.1, Eq. 1) keeps its work arrays on
the stack and on the heap, sized by the number of basis terms: 21 for a quadratic basis in
5D. A driver that includes ``oracle/pcms_oracle.c`` is compiled with ``-fsanitize=address``
and runs fits in 2D-5D at degrees 0, 1 and 2, with and without shape functions, in
brute-force and grid mode and with a Tikhonov term, so that every array the solve writes is
exercised at its largest size. Any out-of-bounds read or write aborts the driver with an
ASan report. No GPU is used.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_C = os.path.join(ROOT, "oracle", "pcms_oracle.c")

DRIVER = r"""
#include "%(src)s"

/* splitmix64: a fixed, seeded sequence of doubles in [0, 1) */
static uint64_t sm_state;
static double urand(void) {
    uint64_t z = (sm_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

int main(void) {
    const double radius[6] = {0, 0, 0.2, 0.3, 0.45, 0.55};
    int bad = 0;
    for (int dim = 2; dim <= 5; dim++) {
        for (int degree = 0; degree <= 2; degree++) {
            for (int variant = 0; variant < 3; variant++) {
                const int64_t ns = 400, nt = 24;
                const int nf = 2;
                sm_state = (uint64_t)(1000 * dim + 10 * degree + variant);
                double* src = (double*)malloc(sizeof(double) * dim * ns);
                double* tgt = (double*)malloc(sizeof(double) * dim * nt);
                double* fld = (double*)malloc(sizeof(double) * nf * ns);
                for (int64_t i = 0; i < dim * ns; i++) src[i] = urand();
                for (int64_t i = 0; i < dim * nt; i++) tgt[i] = 0.2 + 0.6 * urand();
                /* field 0: a polynomial of the basis degree, field 1: noise */
                for (int64_t j = 0; j < ns; j++) {
                    double p = 1.0;
                    for (int d = 0; d < dim; d++) {
                        double x = src[d * ns + j];
                        p += (degree >= 1 ? 0.5 * x : 0.0) + (degree >= 2 ? 0.25 * x * x : 0.0);
                    }
                    fld[j] = p;
                    fld[ns + j] = urand();
                }
                int m = orc_num_terms(dim, degree);
                int need = variant == 2 ? m + 5 : 0;
                int mode = variant == 1 ? 1 : 0;
                double lambda = variant == 2 ? 1e-3 : 0.0;
                int32_t* cnt = (int32_t*)malloc(sizeof(int32_t) * nt);
                int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (nt + 1));
                int32_t* kexp = (int32_t*)malloc(sizeof(int32_t) * nt);
                int64_t nnz = orc_count_neighbors(dim, src, ns, tgt, nt, radius[dim], 0, need,
                                                  mode, cnt, kexp);
                off[0] = 0;
                for (int64_t i = 0; i < nt; i++) off[i + 1] = off[i] + cnt[i];
                if (off[nt] != nnz) bad++;
                int32_t* cols = (int32_t*)malloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1));
                double* shape = (double*)malloc(sizeof(double) * (nnz > 0 ? nnz : 1));
                double* val = (double*)malloc(sizeof(double) * nf * nt);
                int8_t* st = (int8_t*)malloc(nt);
                orc_mls(dim, degree, 0, lambda, src, ns, tgt, nt, fld, nf, radius[dim], need, mode,
                        val, st, kexp, off, cols, shape);
                int nok = 0;
                for (int64_t i = 0; i < nt; i++) {
                    if (st[i] != 0) continue;
                    nok++;
                    if (lambda == 0.0) {
                        double p = 1.0;
                        for (int d = 0; d < dim; d++) {
                            double x = tgt[d * nt + i];
                            p += (degree >= 1 ? 0.5 * x : 0.0) + (degree >= 2 ? 0.25 * x * x : 0.0);
                        }
                        if (!(fabs(val[i] - p) <= 1e-9 * fabs(p))) bad++;
                    }
                }
                printf("dim %%d degree %%d variant %%d: m %%d nnz %%lld ok %%d\n", dim, degree,
                       variant, m, (long long)nnz, nok);
                if (nok == 0) bad++;
                free(src); free(tgt); free(fld); free(cnt); free(off); free(kexp); free(cols);
                free(shape); free(val); free(st);
            }
        }
    }
    printf("bad %%d\n", bad);
    return bad ? 3 : 0;
}
"""


def test_oracle_fits_are_memory_safe_under_asan(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    drv = tmp_path / "asan_driver.c"
    drv.write_text(DRIVER % {"src": ORACLE_C})
    exe = tmp_path / "asan_driver"
    build = subprocess.run(
        ["gcc", "-O1", "-g", "-std=c11", "-fsanitize=address,undefined",
         "-fno-omit-frame-pointer", "-fno-sanitize-recover=all", "-ffp-contract=off",
         "-o", str(exe), str(drv), "-lm"],
        capture_output=True, text=True)
    if build.returncode != 0 and "asan" in (build.stderr or "").lower():
        pytest.skip("AddressSanitizer runtime not available: " + build.stderr[-300:])
    assert build.returncode == 0, build.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0:halt_on_error=1")
    run = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=300)
    report = run.stdout[-2000:] + run.stderr[-4000:]
    assert "AddressSanitizer" not in run.stderr, report
    assert "runtime error" not in run.stderr, report
    assert run.returncode == 0, report
    # every dimension and degree ran, including the 21-term quadratic basis in 5D
    assert "dim 5 degree 2 variant 0: m 21" in run.stdout, report
    assert "dim 4 degree 2 variant 0: m 15" in run.stdout, report
