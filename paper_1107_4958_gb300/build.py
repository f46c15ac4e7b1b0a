"""Builds libgaussbox.so in-tree for sm_103a (nvcc, parallel translation units).

Usage: python -m paper_1107_4958_gb300.build   (or __graft_entry__.build())
"""
import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgaussbox.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
          "-I" + os.path.join(ROOT, "include")]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


# kernel text compiled at run time (NVRTC) and embedded into the library
RUNTIME_KERNELS = {"gb_walker_source": "walker_kernel.cuh", "gb_depth_walker_source": "depth_walker.cuh"}


def _embedded_source():
    """Writes _build/embedded_src.cpp: each run-time kernel's text as a C string."""
    path = os.path.join(OUT_DIR, "embedded_src.cpp")
    parts = ["// generated by build.py from csrc/: kernel text compiled at run time\n"]
    for sym, name in sorted(RUNTIME_KERNELS.items()):
        with open(os.path.join(CSRC, name)) as fh:
            text = fh.read()
        assert ")GBSRC\"" not in text
        parts.append('extern "C" const char %s[] = R"GBSRC(%s)GBSRC";\n' % (sym, text))
    body = "".join(parts)
    if not os.path.exists(path) or open(path).read() != body:
        with open(path, "w") as fh:
            fh.write(body)
    return path


def sources():
    out = []
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cpp")):
            out.append(os.path.join(CSRC, name))
    return out


def _digest():
    h = hashlib.sha256()
    for path in sources() + [os.path.join(CSRC, n) for n in sorted(os.listdir(CSRC)) if n.endswith((".h", ".cuh"))] + \
            [os.path.join(ROOT, "include", "gaussbox.h")]:
        with open(path, "rb") as fh:
            h.update(path.encode() + fh.read())
    h.update(" ".join(ARCH + COMMON).encode())
    return h.hexdigest()


def _compile(src, verbose):
    obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
    cmd = [nvcc()] + ARCH + COMMON + ["-x", "cu" if src.endswith(".cu") else "c++", "-c", src, "-o", obj]
    if verbose and src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stdout))
    return obj, r.stdout


def build(force=False, verbose=False):
    """Compiles every source under csrc/ and links libgaussbox.so.  Returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp = os.path.join(OUT_DIR, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    srcs = sources() + [_embedded_source()]
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose), srcs))
    if verbose:
        for _obj, log in results:
            if log.strip():
                sys.stdout.write(log)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lnvrtc", "-lpthread"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stdout)
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
