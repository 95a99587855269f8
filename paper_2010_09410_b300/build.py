"""Build the CUDA library (sm_103a) in-tree: paper_2010_09410_b300/libtfhe_b300.so."""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libtfhe_b300.so")
LIB_BOUNDS = os.path.join(HERE, "libtfhe_b300_bounds.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def deps():
    return sources() + glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + \
        [os.path.join(os.path.dirname(HERE), "include", "tfhe_b300.h")]


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    """bounds: the debug library libtfhe_b300_bounds.so, compiled with TFHE_BOUNDS_CHECK
    (device index checks that report TFHE_EBOUNDS), in its own object folder."""
    lib = LIB_BOUNDS if bounds else LIB
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(d) <= t for d in deps()):
            return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    objs = []
    build_dir = os.path.join(HERE, "_build_bounds" if bounds else "_build")
    os.makedirs(build_dir, exist_ok=True)
    for src in sources():
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-c", src, "-o", obj]
        if bounds:
            cmd.append("-DTFHE_BOUNDS_CHECK")
        if verbose:
            cmd.append("-Xptxas=-v")
        subprocess.check_call(cmd)
        objs.append(obj)
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", lib, *objs, "-lcudart", "-lcuda"])
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds="--bounds" in sys.argv))
