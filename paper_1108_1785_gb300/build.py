"""Builds the C-ABI library in-tree for sm_103a with nvcc, in two variants from the same
sources:

- libgnm.so          the library;
- libgnm_checked.so  the same with device-side bounds checks (-DGNM_CHECKED=1), which
                     report a failed check as GNM_E_INTERNAL instead of touching memory.

Every .cu/.cpp under csrc/ is compiled to an object in _build/ (_build_checked/), the
translation units of both variants in one parallel pool, the slowest first; then each
variant is linked (CUDA runtime linked statically). Objects are rebuilt when their source
or any header is newer.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
VARIANTS = {  # name: (object folder, library, extra flags)
    "default": (os.path.join(HERE, "_build"), os.path.join(HERE, "libgnm.so"), []),
    "checked": (os.path.join(HERE, "_build_checked"), os.path.join(HERE, "libgnm_checked.so"), ["-DGNM_CHECKED=1"]),
}
LIB = VARIANTS["default"][1]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]
# the template-heavy translation units first (they bound the build's wall time)
SLOW_FIRST = ("agg_rmi", "agg_smem", "agg_radix", "agg_staged", "agg_l2", "agg_hash24", "agg_keys")


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return p


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.hpp")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    return max([os.path.getmtime(h) for h in hs] + [0.0])


def _order(src: str) -> int:
    stem = os.path.splitext(os.path.basename(src))[0]
    return SLOW_FIRST.index(stem) if stem in SLOW_FIRST else len(SLOW_FIRST)


def build(verbose: bool = False, force: bool = False, ptxas_info: bool = False, checked=None) -> str:
    """Builds both variants (checked=None), or only the checked (True) or default (False)
    one; returns the path of the default library (the checked one when checked=True)."""
    names = ["default", "checked"] if checked is None else (["checked"] if checked else ["default"])
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")), key=_order)
    hmt = _headers_mtime()
    cc = nvcc()
    jobs, objs = [], {n: [] for n in names}
    for s in srcs:
        for n in names:
            obj_dir, _, extra = VARIANTS[n]
            os.makedirs(obj_dir, exist_ok=True)
            o = os.path.join(obj_dir, os.path.basename(s) + ".o")
            objs[n].append(o)
            if force or ptxas_info or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hmt):
                cmd = [cc] + ARCH + FLAGS + extra + (["-Xptxas", "-v"] if ptxas_info else []) + ["-c", s, "-o", o]
                if s.endswith(".cpp"):
                    cmd = [cc] + FLAGS + extra + ["-x", "c++", "-c", s, "-o", o]
                jobs.append((s, n, cmd))

    def run(job):
        s, n, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return s, n, r.returncode, r.stdout + r.stderr

    rebuilt = set()
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for s, n, rc, out in ex.map(run, jobs):
                if verbose or rc != 0 or ptxas_info:
                    sys.stderr.write(out)
                if rc != 0:
                    raise RuntimeError(f"nvcc failed on {os.path.basename(s)} ({n} build)")
                rebuilt.add(n)
    for n in names:
        _, lib, _ = VARIANTS[n]
        if n in rebuilt or not os.path.exists(lib):
            tmp = lib + f".{os.getpid()}.tmp"
            cmd = [cc] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs[n] + ["-lpthread"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
                raise RuntimeError(f"link of {os.path.basename(lib)} failed")
            os.replace(tmp, lib)
    return VARIANTS["checked"][1] if checked else LIB


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv, ptxas_info="--ptxas" in sys.argv,
          checked=True if "--checked" in sys.argv else (False if "--default" in sys.argv else None))
    print(LIB)
