"""Build libsdrt.so in-tree: nvcc for sm_103a, translation units compiled in parallel.

Usage: python -m paper_2105_08632_gb300.build   (or build() from Python)
"""
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsdrt.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _nvcc():
    p = os.path.join(CUDA_HOME, "bin", "nvcc")
    return p if os.path.exists(p) else (shutil.which("nvcc") or "nvcc")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _host_cxx():
    return shutil.which("g++") or shutil.which("c++")


def generate(gen_dir):
    """Build and run the operator generator (csrc/gen/opgen.cpp, linked with the
    library's own operator code refel.cpp): one CUDA translation unit per
    specialised element type plus the dispatch table, written to gen_dir."""
    os.makedirs(gen_dir, exist_ok=True)
    exe = os.path.join(BUILD, "opgen")
    srcs = [os.path.join(CSRC, "gen", "opgen.cpp"), os.path.join(CSRC, "refel.cpp")]
    cxx = _host_cxx()
    if cxx:
        cmd = [cxx, "-O1", "-std=c++17", "-I", CSRC, *srcs, "-o", exe]
    else:
        cmd = [_nvcc(), "-O1", "-std=c++17", "-x", "c++", "-I", CSRC, *srcs, "-o", exe]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("operator generator build failed:\n" + r.stdout.decode(errors="replace"))
    for f in os.listdir(gen_dir):
        if f.startswith("gen_"):
            os.remove(os.path.join(gen_dir, f))
    r = subprocess.run([exe, gen_dir], stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("operator generator failed:\n" + r.stdout.decode(errors="replace"))
    return sorted(os.path.join(gen_dir, f) for f in os.listdir(gen_dir) if f.endswith((".cu", ".cpp")))


def build(verbose=False, extra_flags=()):
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    procs, objs = [], []
    for path in _sources() + generate(os.path.join(BUILD, "gen")):
        src = os.path.basename(path)
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if src.endswith(".cu"):
            cmd = [nvcc, "-c", path, "-o", obj, "-std=c++17", "-O3", "-lineinfo", *ARCH,
                   "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-Xptxas", "-v" if verbose else "-O3",
                   *inc, *extra_flags]
        else:
            cmd = [nvcc, "-c", path, "-o", obj, "-std=c++17", "-O2", "-x", "c++", "-Xcompiler", "-fPIC",
                   *inc, *extra_flags]
        procs.append((src, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, cmd, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((src, text))
        elif verbose and text.strip():
            print(f"--- {src}\n{text}")
    if failed:
        msg = "\n".join(f"--- {s}\n{t}" for s, t in failed)
        raise RuntimeError(f"libsdrt build failed:\n{msg}")
    tmp = LIB + ".tmp"
    cmd = [nvcc, "-shared", *ARCH, "-cudart", "static", "-o", tmp, *objs, "-lrt", "-lpthread", "-ldl"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("libsdrt link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
