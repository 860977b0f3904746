"""Builds the conversion library ``libmrn.so`` in-tree with nvcc for sm_103a.

Every ``.cu`` and ``.cpp`` file under ``csrc/`` is compiled into one shared
object next to this file.  ``ptxas -v`` output (registers, spills, shared
memory per kernel) is kept in ``_build/ptxas.log``.
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmrn.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def headers():
    return (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(HERE, "..", "include", "*.h")))


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in sources() + headers())


def _compile(src, obj, log):
    cmd = ["nvcc"] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-Wall",
                             "-Xptxas", "-v", "--expt-relaxed-constexpr", "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    log.write("==== %s\n%s%s" % (os.path.basename(src), r.stdout, r.stderr))
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed on %s" % src)


def build(force=False, jobs=8):
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    objs = []
    from concurrent.futures import ThreadPoolExecutor
    logs = {}
    import io

    def one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        buf = io.StringIO()
        _compile(src, obj, buf)
        logs[src] = buf.getvalue()
        return obj

    with ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(one, sources()))
    with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
        for src in sources():
            f.write(logs.get(src, ""))
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["nvcc"] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
