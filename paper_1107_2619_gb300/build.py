"""Build libmd.so (the CUDA hot path) in-tree with nvcc for sm_103a.

Each .cu file compiles to an object in parallel, then nvcc links the shared library
paper_1107_2619_gb300/_build/libmd.so.  Rebuilds only when a source or header is newer
than the library.  MD_BUILD_VERBOSE=1 adds -Xptxas -v (registers, spills, shared memory).
"""
import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = None, out: str = None, defines=()) -> str:
    """Compile libmd.so (to `out`, default the in-tree _build/libmd.so); `defines` are extra
    -D macros (tuning knobs such as MD_STEP_MIN_BLOCKS)."""
    lib = out or LIB
    if not force and out is None and not _stale():
        return LIB
    verbose = os.environ.get("MD_BUILD_VERBOSE") == "1" if verbose is None else verbose
    obj_dir = os.path.join(os.path.dirname(lib), "obj")
    os.makedirs(obj_dir, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if verbose:
        flags += ["-Xptxas", "-v"]
    flags += [f"-D{d}" for d in defines]

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        r = subprocess.run(["nvcc", "-c", src, "-o", obj] + flags, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, _sources()))
    if verbose:
        for _, log in results:
            print(log)
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run(["nvcc", "-shared"] + ARCH + ["-o", tmp] + [o for o, _ in results],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
