"""Build the in-tree shared library libsvgb300.so (CUDA sm_103a + host C++).

Every translation unit is compiled in parallel; CUDA sources with
``nvcc -gencode arch=compute_103a,code=sm_103a -lineinfo``.  No cmake.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libsvgb300.so")
BUILD = os.path.join(HERE, "_build")


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(nv))
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


# stage_inst.cu is compiled once per (precision, direction, register width): the
# stage-sweep instantiations are the bulk of the device code, so they build in parallel.
STAGE_INST = ([("float", 1, r) for r in range(1, 6)] + [("float", 2, r) for r in range(1, 5)] +
              [("double", 1, r) for r in range(1, 5)] + [("double", 2, r) for r in range(1, 4)])


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def units():
    """(source file, object name, extra defines) of every translation unit."""
    out = []
    for f in sources():
        if f == "stage_inst.cu":
            for real, nv, r in STAGE_INST:
                out.append((f, f"stage_inst_{real}_nv{nv}_r{r}.o",
                            [f"-DSVK_INST_REAL={real}", f"-DSVK_INST_NV={nv}", f"-DSVK_INST_R={r}"]))
        else:
            out.append((f, f + ".o", []))
    return out


def _embed_prelude():
    """jit_prelude.cuh as a C++ string constant: the run-time compiled stage kernels
    include it from memory (NVRTC gets no include path)."""
    src = open(os.path.join(CSRC, "jit_prelude.cuh")).read()
    assert ")SVJIT\"" not in src
    text = ("// generated by build.py from csrc/jit_prelude.cuh\n#pragma once\n"
            "static const char kJitPrelude[] = R\"SVJIT(" + src + ")SVJIT\";\n")
    out = os.path.join(BUILD, "jit_prelude_inc.h")
    if not os.path.exists(out) or open(out).read() != text:
        with open(out, "w") as f:
            f.write(text)


def build(verbose=False, force=False):
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(BUILD, exist_ok=True)
    _embed_prelude()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", BUILD]
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "sv.h"))
    newest_header = max(os.path.getmtime(h) for h in headers)
    jobs = []
    objs = []
    for f, oname, defs in units():
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, oname)
        objs.append(obj)
        if (not force and os.path.exists(obj)
                and os.path.getmtime(obj) >= max(os.path.getmtime(src), newest_header)):
            continue
        if f.endswith(".cu"):
            cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3",
                   "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                   "-Xptxas", "-v" if verbose else "-O3", "-c", src, "-o", obj] + defs + inc
        else:
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function",
                   "-I", os.path.join(cuda, "include"), "-c", src, "-o", obj] + inc
        jobs.append(cmd)
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
            outs = list(ex.map(_run, jobs))
        if verbose:
            for o in outs:
                sys.stdout.write(o)
    if jobs or not os.path.exists(OUT):
        _run([nvcc, "-shared", "-o", OUT] + objs + ["-cudart", "shared",
              "-L", os.path.join(cuda, "lib64"), "-lnvrtc", "-Xlinker", "-rpath," + os.path.join(cuda, "lib64")])
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
