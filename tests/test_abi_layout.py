"""The ctypes mirrors of the C-ABI (no GPU): a small C program, compiled with the host compiler
against include/helm.h, prints every struct field's offset and size and every enum value; the
Python binding's structures and constants must agree with them exactly."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "helm_grid": ("_Grid", ["dim", "n", "lo", "hi"]),
    "helm_mg_params": ("_MG", ["kind", "theta_a", "beta1", "beta2", "re_lambda0", "nu1", "nu2", "omega",
                               "smoother", "gamma_f", "gamma_c", "coarsest_n", "prec", "gs_arith"]),
    "helm_stats": ("_Stats", ["iterations", "restarts", "status", "rel_res", "est_res", "time_ms", "history",
                              "history_len", "reorthogonalizations"]),
    "helm_tuning": ("_Tuning", ["tail_levels", "level_tile", "cluster_levels", "cluster_ctas", "cluster_halo"]),
}
ENUMS = ["HELM_OK", "HELM_ERR_ARG", "HELM_ERR_CUDA", "HELM_ERR_NOMEM", "HELM_ERR_NOCONV", "HELM_ERR_BREAKDOWN",
         "HELM_ERR_NONFINITE", "HELM_ERR_TIMEOUT", "HELM_C128", "HELM_C64", "HELM_PC_NONE", "HELM_PC_CSG",
         "HELM_PC_CSL", "HELM_PC_QD", "HELM_PC_LAPLACE", "HELM_OP_A", "HELM_OP_M", "HELM_FGMRES", "HELM_BICGSTAB",
         "HELM_SMOOTH_JACOBI", "HELM_SMOOTH_RB", "HELM_GS_FP64", "HELM_GS_DF", "HELM_GS_DCGS2", "HELM_MAX_LEVELS"]
TILES = {"none": "HELM_TILE_NONE", "32x8": "HELM_TILE_32x8", "16x16": "HELM_TILE_16x16", "16x8": "HELM_TILE_16x8",
         "64x4": "HELM_TILE_64x4", "wave": "HELM_TILE_WAVE", "8x8": "HELM_TILE_8x8"}
ENGINES = {"auto": "HELM_BATCH_AUTO", "lockstep": "HELM_BATCH_LOCKSTEP", "streams": "HELM_BATCH_STREAMS"}
CLASSES = ["HELM_K_APPLY", "HELM_K_SMOOTH_FINE", "HELM_K_SMOOTH_COARSE", "HELM_K_RESTRICT", "HELM_K_PROLONG",
           "HELM_K_COARSE", "HELM_K_MDOT", "HELM_K_UPDATE_MDOT", "HELM_K_UPDATE_NORM", "HELM_K_VECTOR", "HELM_K_SMALL"]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "helm.h"', "int main(void) {"]
    for s, (_, fields) in STRUCTS.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (s, s))
        for f in fields:
            lines.append('printf("%s.%s %%zu %%zu\\n", offsetof(%s, %s), sizeof(((%s *)0)->%s));' % (s, f, s, f, s, f))
    for e in ENUMS + list(TILES.values()) + list(ENGINES.values()) + CLASSES + ["HELM_K_NCLASS", "HELM_TILE_COUNT"]:
        lines.append('printf("%s %%d\\n", (int)(%s));' % (e, e))
    lines += ["return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        k, *v = line.split()
        table[k] = tuple(int(x) for x in v)
    return table


@pytest.fixture(scope="module")
def binding():
    from paper_1012_4307_gb300 import helm
    return helm


def test_struct_layouts_match(c_layout, binding):
    for s, (py, fields) in STRUCTS.items():
        cls = getattr(binding, py)
        assert C.sizeof(cls) == c_layout[s][0], s
        assert [f[0] for f in cls._fields_] == fields, s
        for f in fields:
            desc = getattr(cls, f)
            assert (desc.offset, desc.size) == c_layout["%s.%s" % (s, f)], (s, f)


def test_enum_values_match(c_layout, binding):
    for e in ENUMS:
        assert getattr(binding, e) == c_layout[e][0], e
    for name, e in TILES.items():
        assert binding.TILES[name] == c_layout[e][0], name
    assert len(binding.TILES) == c_layout["HELM_TILE_COUNT"][0] + 1  # the shapes and "none"
    for name, e in ENGINES.items():
        assert binding.BATCH_ENGINES[name] == c_layout[e][0], name
    assert len(binding.KERNEL_CLASSES) == c_layout["HELM_K_NCLASS"][0]
    for i, e in enumerate(CLASSES):
        assert c_layout[e][0] == i
