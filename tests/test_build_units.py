"""The build compiles every CUDA translation unit of the library: each
`*.cu` file under paper_2203_09467_gb300/csrc is a unit of build.py (the
FP64 ones with --fmad=false), and each Launch member is instantiated in
exactly one of the kernel units."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2203_09467_gb300", "csrc")


def test_every_cu_file_is_built():
    from paper_2203_09467_gb300 import build
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    assert sorted(build.UNITS) == cu
    for name, flags in build.UNITS.items():
        if "fp64" in name or name == "emt_tables.cu":
            assert "--fmad=false" in flags, name


def test_each_kernel_family_instantiated_once_per_precision():
    macros = {}
    for f in os.listdir(CSRC):
        if f.startswith("emt_kernels_") and f.endswith(".cu"):
            for m in re.findall(r"^(EMT_INSTANTIATE_\w+)\((\w+)\)", open(os.path.join(CSRC, f)).read(), re.M):
                macros.setdefault(m, []).append(f)
    fams = ("FUSED", "PERSIST", "SPLIT", "PIPE")
    assert sorted(macros) == sorted((f"EMT_INSTANTIATE_{fam}", r) for fam in fams for r in ("double", "float"))
    assert all(len(v) == 1 for v in macros.values()), macros
