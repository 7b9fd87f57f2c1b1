"""Build libmm_b300.so in-tree with nvcc for sm_103a (B300).

    python -m paper_1501_07293_b300.build [--verbose] [--ptxas-info] [--bounds-check]

Each .cu file under csrc/ is compiled to an object in parallel, then linked
into ``paper_1501_07293_b300/libmm_b300.so`` (``--bounds-check``: the
bounds-check build ``libmm_b300_bc.so``, compiled with -DMM_BOUNDS_CHECK).
Rebuilds only when a source or header is newer than the library.
"""
import argparse
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libmm_b300.so")
OBJDIR = os.path.join(ROOT, "_build")
# the bounds-check build (-DMM_BOUNDS_CHECK): the same library with index checks
# in the kernels that report to a device flag instead of trapping
LIB_BC = os.path.join(PKG, "libmm_b300_bc.so")
OBJDIR_BC = os.path.join(ROOT, "_build", "bc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-diag-suppress", "128",
         "-Xcompiler", "-O2", "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    # the y/z instantiation units take longest: start them first
    def cost(path):
        name = os.path.basename(path)
        return (0 if name.startswith("field_inst_yz") else 1 if name.startswith("field_inst") else 2, name)
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")), key=cost)


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)])


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force=False, verbose=False, ptxas_info=False, bounds_check=False):
    lib_out = LIB_BC if bounds_check else LIB
    objdir = OBJDIR_BC if bounds_check else OBJDIR
    if not force and up_to_date(lib_out):
        return lib_out
    nvcc = _nvcc()
    os.makedirs(objdir, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    if bounds_check:
        extra += ["-DMM_BOUNDS_CHECK"]

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, (r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(compile_one, _sources()))
    if verbose or ptxas_info:
        for _, log in results:
            if log.strip():
                print(log)
    tmp = lib_out + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_out)
    return lib_out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true")
    ap.add_argument("--bounds-check", action="store_true", help="build libmm_b300_bc.so (-DMM_BOUNDS_CHECK)")
    a = ap.parse_args(argv)
    print(build(force=a.force or a.ptxas_info, verbose=a.verbose, ptxas_info=a.ptxas_info,
                bounds_check=a.bounds_check))


if __name__ == "__main__":
    sys.exit(main())
