"""Build libpff.so (sm_103a) in-tree with nvcc: kernel translation units per
precision compiled in parallel, then linked with the C-ABI host code."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpff.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-O3"]

KERNEL_TUS = ["k_rowfwd.cu", "k_rowinv.cu", "k_col.cu", "k_elem.cu"]
PRECISIONS = {"f32": "float", "f64": "double"}


def nvcc():
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpff")


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))] + \
        [os.path.join(HERE, "..", "include", "pff.h")]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources()) or os.path.getmtime(__file__) > t


def build(force=False, verbose=False, jobs=None):
    """Compile (if sources changed) and return the path of libpff.so."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    jobs_list = []
    for tu in KERNEL_TUS:
        for tag, real in PRECISIONS.items():
            obj = os.path.join(BUILD, tu.replace(".cu", f"_{tag}.o"))
            jobs_list.append([cc, *ARCH, *FLAGS, f"-DPFF_REAL={real}", "-c", os.path.join(CSRC, tu), "-o", obj])
    for host_tu in ("api.cu", "noalloc.cu", "micro.cu"):
        jobs_list.append([cc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, host_tu),
                          "-o", os.path.join(BUILD, host_tu.replace(".cu", ".o"))])
    # the cluster mechanics solve (FP32 only)
    jobs_list.append([cc, *ARCH, *FLAGS, "-DPFF_REAL=float", "-c", os.path.join(CSRC, "k_cluster.cu"),
                      "-o", os.path.join(BUILD, "k_cluster.o")])
    # persistent kernels: their blocks read what other blocks of the same launch wrote,
    # so global loads bypass L1 (-dlcm=cg) and 8-byte staging copies use L2-only loads
    jobs_list.append([cc, *ARCH, *FLAGS, "-DPFF_REAL=float", "-DPFF_L2_ONLY", "-Xptxas", "-dlcm=cg", "-c",
                      os.path.join(CSRC, "k_persist.cu"), "-o", os.path.join(BUILD, "k_persist.o")])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return cmd[-1]

    n = jobs or max(1, min(len(jobs_list), os.cpu_count() or 4))
    with ThreadPoolExecutor(n) as ex:
        objs = list(ex.map(run, jobs_list))
    tmp = LIB + ".tmp"
    link = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    t = __import__("time").time()
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
    print("seconds", round(__import__("time").time() - t, 1))
