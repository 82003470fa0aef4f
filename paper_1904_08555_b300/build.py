"""Build libcj.so in-tree for sm_103a.

Steps: embed the kernel template sources as C++ string literals (the
in-memory files NVRTC compiles from), compile the AoT kernel unit with nvcc,
compile the host library with g++, and link everything with the static NVRTC,
nvptxcompiler and CUDA runtime libraries so that run-time compilation opens
no file.  Only the cj_* symbols are exported.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
KDIR = os.path.join(CSRC, "kernels")
GEN = os.path.join(CSRC, "generated")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcj.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

EMBEDDED = [("cj_emb_geometry_h", "geometry.h"),
            ("cj_emb_update_chain_cuh", "update_chain.cuh"),
            ("cj_emb_ltimes_cuh", "ltimes.cuh"),
            ("cj_emb_mass_cuh", "mass.cuh"),
            ("cj_emb_chain_tc_cuh", "chain_tc.cuh")]


def _sources():
    srcs = [os.path.join(CSRC, f) for f in ("cj.cpp", "aot.cu", "noalloc.cu", "tuner.cu", "cj_internal.h")]
    srcs += [os.path.join(KDIR, "mlp.cuh")]
    srcs += [os.path.join(KDIR, f) for _, f in EMBEDDED]
    srcs += [os.path.join(ROOT, "include", "cj.h"), __file__]
    return srcs


def _embed():
    os.makedirs(GEN, exist_ok=True)
    parts = ["// generated by build.py from csrc/kernels -- do not edit\n"]
    for var, fname in EMBEDDED:
        with open(os.path.join(KDIR, fname)) as f:
            text = f.read()
        assert ")CJEMBED\"" not in text
        parts.append(f'static const char {var}[] = R"CJEMBED({text})CJEMBED";\n')
    path = os.path.join(GEN, "embedded_sources.inc")
    new = "".join(parts)
    if not os.path.exists(path) or open(path).read() != new:
        with open(path, "w") as f:
            f.write(new)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("build step failed: " + " ".join(cmd[:3]))
    return r


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    _embed()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", os.path.join(CUDA, "include")]
    _run([os.path.join(CUDA, "bin", "nvcc"), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
          "-Xcompiler", "-fvisibility=hidden", *inc, "-c", os.path.join(CSRC, "aot.cu"),
          "-o", os.path.join(OUT, "aot.o")])
    for unit in ("noalloc", "tuner"):
        _run([os.path.join(CUDA, "bin", "nvcc"), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", *inc, "-c", os.path.join(CSRC, unit + ".cu"),
              "-o", os.path.join(OUT, unit + ".o")])
    _run(["g++", "-O2", "-std=c++17", "-fPIC", "-fvisibility=hidden", "-Wall", *inc, "-c",
          os.path.join(CSRC, "cj.cpp"), "-o", os.path.join(OUT, "cj.o")])
    ver = os.path.join(OUT, "exports.map")
    with open(ver, "w") as f:
        f.write("{ global: cj_*; local: *; };\n")
    lib64 = os.path.join(CUDA, "lib64")
    tmp = LIB + ".tmp"
    _run(["g++", "-shared", "-o", tmp, os.path.join(OUT, "aot.o"), os.path.join(OUT, "noalloc.o"),
          os.path.join(OUT, "tuner.o"), os.path.join(OUT, "cj.o"),
          "-L" + lib64, "-Wl,--start-group", "-lnvrtc_static", "-lnvrtc-builtins_static",
          "-lnvptxcompiler_static", "-Wl,--end-group", "-lcudart_static", "-lpthread", "-ldl", "-lrt",
          "-Wl,--exclude-libs,ALL", "-Wl,--version-script=" + ver, "-Wl,--gc-sections", "-s"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
