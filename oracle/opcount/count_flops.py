"""Algorithmic FP64 flops per cell of the oracle's sweeps and CFL pass.

TEST INFRASTRUCTURE ONLY (an op-counting build of the oracle).  The script
rewrites oracle/ppmlr_oracle.c mechanically into C++ in which every double is
a counting type (counting_double.hpp), with one change of accounting: the PPM
slope and interface coefficients depend only on the widths, not on the
reconstructed variable, so they are charged once per zone (for the first of
the seven reconstructed variables) -- the per-variable work is counted for
all seven.  Each +, -, x, /, sqrt is one flop; comparisons are not flops.

    python oracle/opcount/count_flops.py [nx ny nz]

builds _build/liborc_count.so beside this file (no OpenMP: the counters are
global) and prints, on the magnetosphere workload (256 x 192 x 192, finest
spacing 0.4 R_E, by default), the flops per interior cell of the CFL pass and
of one sweep per axis.
"""
import ctypes
import os
import re
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
SRC = os.path.join(ROOT, "oracle", "ppmlr_oracle.c")
OUT = os.path.join(HERE, "_build")

# the coefficient parts of the PPM slope and interface formulas, restated
# with the coefficients named so that they can be charged once per zone
PATCHES = [
    ("""    double s3 = xi[i - 1] + xi[i] + xi[i + 1];
    return xi[i] / s3 * ((2.0 * xi[i - 1] + xi[i]) / (xi[i + 1] + xi[i]) * dp
                         + (xi[i] + 2.0 * xi[i + 1]) / (xi[i - 1] + xi[i]) * dm);""",
     """    mute();
    double s3 = xi[i - 1] + xi[i] + xi[i + 1];
    double c1 = xi[i] / s3, c2 = (2.0 * xi[i - 1] + xi[i]) / (xi[i + 1] + xi[i]);
    double c3 = (xi[i] + 2.0 * xi[i + 1]) / (xi[i - 1] + xi[i]);
    unmute();
    return c1 * (c2 * dp + c3 * dm);"""),
    ("""    double z1 = (x0 + x1) / (2.0 * x1 + x2);
    double z2 = (x3 + x2) / (2.0 * x2 + x1);
    double d = a[i + 1] - a[i];
    double s4 = x0 + x1 + x2 + x3;
    return a[i] + x1 / (x1 + x2) * d
           + 1.0 / s4 * (2.0 * x2 * x1 / (x1 + x2) * (z1 - z2) * d
                         - x1 * z1 * dmi1 + x2 * z2 * dmi);""",
     """    mute();
    double z1 = (x0 + x1) / (2.0 * x1 + x2);
    double z2 = (x3 + x2) / (2.0 * x2 + x1);
    double s4 = x0 + x1 + x2 + x3;
    double k1 = x1 / (x1 + x2), k2 = 1.0 / s4, k3 = 2.0 * x2 * x1 / (x1 + x2) * (z1 - z2);
    double k4 = x1 * z1, k5 = x2 * z2;
    unmute();
    double d = a[i + 1] - a[i];
    return a[i] + k1 * d + k2 * (k3 * d - k4 * dmi1 + k5 * dmi);"""),
    ("""    for (int v = 0; v < NREC; v++) orc_ppm_edges(NP, dm, b->q[v], 1, b->edge[v]);""",
     """    for (int v = 0; v < NREC; v++) { g_coef = v == 0; orc_ppm_edges(NP, dm, b->q[v], 1, b->edge[v]); }
    g_coef = 1;"""),
    ("""        orc_ppm_edges(n4, b->dxL + 4, b->rq[v] + 4, 1, b->edge[v] + 4);""",
     """        g_coef = v == 0;
        orc_ppm_edges(n4, b->dxL + 4, b->rq[v] + 4, 1, b->edge[v] + 4);
        g_coef = 1;"""),
]

PROLOGUE = """#include "counting_double.hpp"
OpCount g_ops;
static int g_coef = 1;                 // 0: coefficient work of this call is not charged
static OpCount g_saved;
static void mute() { if (!g_coef) g_saved = g_ops; }
static void unmute() { if (!g_coef) g_ops = g_saved; }
extern "C" {
void orc_ops(long long *out)
{
    out[0] = g_ops.add; out[1] = g_ops.mul; out[2] = g_ops.div; out[3] = g_ops.sqrt_; out[4] = g_ops.cmp;
}
"""


def build():
    src = open(SRC).read()
    for old, new in PATCHES:
        assert src.count(old) == 1, "the oracle changed: update the op-counting patches\n" + old
        src = src.replace(old, new)
    src = re.sub(r"\bdouble\b", "cdouble", src)
    src = src.replace("#include <string.h>\n", "#include <string.h>\n" + PROLOGUE, 1)
    src += "\n}  // extern \"C\"\n"
    os.makedirs(OUT, exist_ok=True)
    cpp = os.path.join(OUT, "orc_count.cpp")
    lib = os.path.join(OUT, "liborc_count.so")
    open(cpp, "w").write(src)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-I", HERE,
                           "-o", lib, cpp])
    return lib


def main():
    lib = build()
    os.environ["PPMLR_ORACLE_LIB"] = lib
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1607_02214_gb300 import inputs
    L = oracle.lib()
    L.orc_ops.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
    buf = (ctypes.c_longlong * 5)()

    def snap():
        L.orc_ops(buf)
        return list(buf)

    n = tuple(int(x) for x in sys.argv[1:4]) if len(sys.argv) > 3 else (256, 192, 192)
    pr = inputs.magnetosphere(n=n, h0=0.4 * 256 / n[0])
    bc = pr.bc
    o = oracle.Oracle(pr.edges, pr.gamma, bc.flat_faces(), inflow=bc.inflow, dipole_moment=bc.dipole_moment,
                      r_inner=bc.r_inner, inner=bc.inner, p_min=bc.p_min, powell=bc.powell)
    o.set_state(pr.U0)
    cells = pr.cells

    def per_cell(a, b):
        d = [(y - x) / cells for x, y in zip(a, b)]
        return {"add": d[0], "mul": d[1], "div": d[2], "sqrt": d[3], "flops": sum(d[:4]), "cmp": d[4]}

    s0 = snap()
    dt = o.cfl_dt(pr.cfl)
    print("cfl", {k: round(v, 1) for k, v in per_cell(s0, snap()).items()})
    for axis in range(3):
        s0 = snap()
        o.sweep(axis, dt)
        print("sweep", "xyz"[axis], {k: round(v, 1) for k, v in per_cell(s0, snap()).items()})


if __name__ == "__main__":
    main()
