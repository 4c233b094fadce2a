"""Build libcrac.so (the product) and libcrac_testkit.so (test mutators).

nvcc compiles each translation unit for sm_103a only, in parallel, and links
them into shared libraries under paper_2008_10596_gb300/_lib/ (git-ignored;
rebuilt on every machine).
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")
LIB_DIR = os.path.join(PKG, "_lib")
OBJ_DIR = os.path.join(PKG, "_build")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
          "-I", INC, "-I", CSRC] + ARCH

LIBS = {
    "libcrac.so": ["crac_pass_split.cu", "crac_pass_fused.cu", "crac_pass_tma.cu", "crac_pass_per_alloc.cu",
                   "crac_restore.cu", "crac_codec.cu", "crac_noalloc.cu", "crac_drain.cu", "crac_arena.cpp", "crac_image.cpp", "crac_pass.cpp", "crac_restart.cpp",
                   "crac_tune.cpp", "crac_server.cpp", "crac_abi.cpp"],
    "libcrac_testkit.so": ["crac_testkit.cu"],
}


def _deps_newer(target, sources):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    extra = [os.path.join(INC, "crac.h"), os.path.join(CSRC, "crac_kernels.cuh"),
             os.path.join(CSRC, "crac_device.cuh"), os.path.join(CSRC, "crac_codec.cuh"),
             os.path.join(CSRC, "crac_runtime.h")]
    return any(os.path.getmtime(s) > t for s in list(sources) + extra)


def _compile(src, extra=()):
    os.makedirs(OBJ_DIR, exist_ok=True)
    obj = os.path.join(OBJ_DIR, os.path.basename(src) + ".o")
    if not _deps_newer(obj, [src]):
        return obj
    lang = ["-x", "cu"] if src.endswith(".cu") else ["-x", "c++"]
    cmd = [NVCC] + COMMON + list(extra) + lang + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose: bool = False, ptxas_info: bool = False) -> dict:
    os.makedirs(LIB_DIR, exist_ok=True)
    srcs = sorted({s for v in LIBS.values() for s in v})
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = dict(zip(srcs, ex.map(lambda s: _compile(os.path.join(CSRC, s), extra), srcs)))
    out = {}
    for lib, parts in LIBS.items():
        target = os.path.join(LIB_DIR, lib)
        deps = [objs[p] for p in parts]
        if _deps_newer(target, deps):
            tmp = target + f".tmp{os.getpid()}"
            cmd = [NVCC, "-shared"] + ARCH + deps + ["-o", tmp]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed for {lib}:\n{r.stdout}\n{r.stderr}")
            os.replace(tmp, target)
        out[lib] = target
        if verbose:
            print(target)
    return out


if __name__ == "__main__":
    build(verbose=True, ptxas_info="-v" in sys.argv)
