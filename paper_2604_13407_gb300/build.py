"""Build the CUDA library liblbm.so in-tree (paper_2604_13407_gb300/_lib/).

Each translation unit is compiled for sm_103a only, in parallel, and linked with
nvcc.  The FP64 kernels are compiled without fused multiply-add contraction so that
the FP64 path rounds like a plain evaluation of the same expressions; the FP32-arithmetic
kernels use the hardware reciprocal and square root.
"""
import concurrent.futures
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "liblbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
          "-Xcompiler", "-ffp-contract=off",
          "--expt-relaxed-constexpr"]
# FP32 arithmetic (FP32/FP16/BF16 storage) uses the hardware reciprocal and square root
# (relative error ~2^-22, far below the FP32 tolerances); FP64 keeps IEEE division and
# square root and no multiply-add contraction.
FAST32 = ["-prec-div=false", "-prec-sqrt=false"]
UNITS = {
    "lbm_api.cu": [],
    "lbm_adjoint.cu": [],
    "k_f64.cu": ["-fmad=false"],
    "k_f32.cu": FAST32,
    "k_f16.cu": FAST32,
    "k_bf16.cu": FAST32,
    "lbm_noalloc.cu": FAST32,
    "lbm_lbana.cu": [],
}


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cuh", ".h"))) + [os.path.join(HERE, "..", "include", "lbm.h")]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link liblbm.so if it is missing or older than a source."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")

    def compile_one(item):
        name, extra = item
        obj = os.path.join(OUT, name.replace(".cu", ".o"))
        defs = os.environ.get("LBM_NVCC_DEFS", "").split()  # e.g. "-DLBM_F32_IEEE=1"
        cmd = [nvcc] + ARCH + COMMON + extra + defs + ["-c", os.path.join(CSRC, name), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (name, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, UNITS.items()))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
