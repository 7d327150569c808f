"""In-tree build of the CUDA library ``_build/liblbm_gb300.so`` for sm_103a.

The three translation units (one per lattice plus the host ABI) are compiled
in parallel with nvcc and linked into one shared library with the CUDA
runtime linked dynamically (so a process that already loaded libcudart from
PyTorch uses the same runtime).  Also regenerates nothing: the lattice tables
are committed and only rewritten by ``csrc/gen_tables.py``.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbm_gb300.so")
SOURCES = ["lbm_d2q37.cu", "lbm_d3q39.cu", "lbm_abi.cu", "lbm_static.cu", "lbm_batch.cu"]
HEADERS = ["lbm_device.cuh", "lbm_kernels.cuh", "lbm_launch.cuh", "lbm_tma.cuh", "lbm_batch.cuh",
           "lbm_async.cuh", "lbm_wave.cuh", "lbm_df.cuh", "lbm_ctx.h", "lattice_tables.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _cuda_lib_dir():
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(
        subprocess.check_output(["which", _nvcc()]).decode().strip()))), "lib64")


def flags():
    """nvcc flags; LBM_NVCC_DEFINES (e.g. "LBM_FLOAT_D2Q37_BLOCKS=4") adds -D
    tuning definitions for experiments."""
    extra = [f"-D{d}" for d in os.environ.get("LBM_NVCC_DEFINES", "").split() if d]
    return ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                   "-I", os.path.join(os.path.dirname(HERE), "include")] + extra


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile (if needed) and return the path of liblbm_gb300.so."""
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [
        os.path.join(os.path.dirname(HERE), "include", "lbm.h")]
    procs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [_nvcc()] + flags() + ["-c", s, "-o", o + ".tmp"]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), o))
    errs = []
    for p, o in procs:
        out, _ = p.communicate()
        if p.returncode:
            errs.append(out.decode(errors="replace"))
        else:
            os.replace(o + ".tmp", o)
    if errs:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    if force or _stale(LIB, objs):
        libdir = _cuda_lib_dir()
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [_nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
            "-Xlinker", f"-rpath,{libdir}"]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
