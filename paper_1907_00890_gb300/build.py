"""Build the sm_103a shared library ``_lib/libvofp.so`` in-tree with nvcc (no CMake, no torch extension).

Each ``csrc/*.cu`` translation unit is compiled in parallel to ``_build/*.o`` and linked with the shared CUDA
runtime so that the library and PyTorch use one runtime instance.  Rebuilds only when a source or header is
newer than the library.  ``build(checked=True)`` makes the bounds-checked variant ``_lib/libvofp_checked.so``
(``-DVOFP_CHECKED``, objects in ``_build_checked/``), which the binding loads instead when the environment
sets ``VOFP_CHECKED=1``; ``build_all()`` compiles both at once.
"""
import concurrent.futures
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libvofp.so")
LIB_CHECKED = os.path.join(LIBDIR, "libvofp_checked.so")
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _cuda_lib_dir(nvcc):
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def lib_path(checked=False):
    return LIB_CHECKED if checked else LIB


def up_to_date(checked=False):
    lib = lib_path(checked)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def build(force=False, verbose=False, extra_flags=(), checked=False):
    """Compile and link; returns the library path."""
    lib = lib_path(checked)
    if not force and up_to_date(checked):
        return lib
    nvcc = _nvcc()
    objdir = BUILD_CHECKED if checked else BUILD
    os.makedirs(objdir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC,
                     "--expt-relaxed-constexpr"] + (["-DVOFP_CHECKED"] if checked else []) + list(extra_flags)

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc] + common + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    srcs = sources()
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "--cudart", "shared", "-o", tmp] + objs + \
        ["-Xlinker", "-rpath=" + _cuda_lib_dir(nvcc)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib)
    return lib


def build_all(force=False, verbose=False):
    """The plain and the bounds-checked library, compiled concurrently; returns both paths."""
    with concurrent.futures.ThreadPoolExecutor(max_workers=2) as ex:
        futs = [ex.submit(build, force, verbose, (), c) for c in (False, True)]
        return [f.result() for f in futs]


if __name__ == "__main__":
    print(build(force=True, verbose=True))
