"""Build liblbx.so (the C-ABI library) in-tree for sm_103a with nvcc.

Usage: python paper_2607_05668_b300/build.py [--verbose] [--ptxas-info]
Each .cu under csrc/ is compiled to an object in _build/ (in parallel, only when its
sources changed), then linked into paper_2607_05668_b300/liblbx.so.
"""
import argparse
import concurrent.futures as cf
import glob
import hashlib
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
OUT = os.path.join(PKG, "liblbx.so")
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _digest(paths, extra):
    h = hashlib.sha256()
    for p in sorted(paths):
        h.update(open(p, "rb").read())
    h.update(" ".join(extra).encode())
    return h.hexdigest()


def build(verbose=False, ptxas_info=False, jobs=None):
    os.makedirs(BUILD, exist_ok=True)
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    flags = ARCH + FLAGS + (["-Xptxas", "-v"] if ptxas_info else [])

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        stamp = obj + ".sha"
        dig = _digest([src] + headers, flags)
        if os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == dig and not ptxas_info:
            return obj, ""
        cmd = [NVCC] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        open(stamp, "w").write(dig)
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=jobs or os.cpu_count()) as ex:
        results = list(ex.map(compile_one, sources))
    for _, log in results:
        if verbose and log:
            print(log)
    objs = [o for o, _ in results]
    link = [NVCC] + ARCH + ["-shared", "-o", OUT] + objs + ["-cudart", "static"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return OUT


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true")
    a = ap.parse_args()
    print(build(a.verbose, a.ptxas_info))
