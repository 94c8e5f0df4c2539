"""Build libgrafx.so (the C-ABI library) in-tree for sm_103a with nvcc.

    python -m paper_2408_03204_b300.build
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
# GRAFX_VARIANT=precise builds libgrafx_precise.so: the compressor's per-sample gain path
# with correctly rounded ln / exp and IEEE division instead of the hardware
# approximations (a measurement build; the package loads it under the same variable).
VARIANT = os.environ.get("GRAFX_VARIANT", "")
VARIANTS = {"": ("libgrafx.so", "_build", []),
            "precise": ("libgrafx_precise.so", "_build_precise", ["-DGRAFX_PRECISE_GAIN"])}
LIB_NAME, OBJDIR, VARIANT_FLAGS = VARIANTS[VARIANT]
LIB = os.path.join(HERE, LIB_NAME)
SOURCES = ["capi.cu", "k_elem.cu", "k_eq.cu", "k_comp.cu", "k_loss.cu", "k_optim.cu", "k_delay.cu", "k_reverb.cu", "k_warm.cu", "k_bal.cu", "plan.cpp", "schedule.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    for d in (CSRC, os.path.join(HERE, "..", "include")):
        for f in os.listdir(d):
            if os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return False


def build(force=False, verbose=False, jobs=None):
    if not force and not needs_build():
        return LIB
    objdir = os.path.join(HERE, OBJDIR)
    os.makedirs(objdir, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xptxas", "-O3"] + VARIANT_FLAGS
    procs, objs = [], []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(objdir, s + ".o")
        objs.append(obj)
        cmd = [nvcc()] + common + ["-c", src, "-o", obj]
        if s.endswith(".cpp"):
            cmd = [nvcc(), "-x", "c++", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errs = []
    for s, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0 or verbose:
            errs.append(f"--- {s}\n{out.decode()}")
        if pr.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    link = [nvcc()] + ARCH + ["-shared", "-o", LIB] + objs + ["-cudart", "static", "-lpthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode())
    if verbose and errs:
        print("\n".join(errs))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
