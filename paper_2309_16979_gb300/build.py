"""Build the C-ABI library libsvgb300.so in-tree with nvcc for sm_103a.

Each translation unit compiles in parallel (one -gencode, no cmake), then one
nvcc link produces the shared library next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "libsvgb300.so")
BUILD = os.path.join(HERE, "_build")

SOURCES = ["codec.cu", "apply.cu", "apply_phase.cu", "reduce.cu", "noalloc.cu", "plan.cpp", "engine.cpp", "api.cpp",
           "jit.cpp", "transfer.cu"]
# device headers embedded into the library for the kernels it generates and
# compiles at run time (jit.cpp)
JIT_HEADERS = ["sv_dev_types.h", "codec_dev.cuh", "tile_dev.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _flags():
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
            "-I", INCLUDE, "-I", CSRC, "-I", BUILD] + ARCH


def _write_jit_embed() -> str:
    """Write _build/jit_embed.inc: the JIT device headers as raw string
    literals (rewritten only when their text changes)."""
    path = os.path.join(BUILD, "jit_embed.inc")
    parts = ["// generated by build.py from " + ", ".join(JIT_HEADERS) + "\n"]
    names, texts = [], []
    for i, h in enumerate(JIT_HEADERS):
        text = open(os.path.join(CSRC, h)).read()
        tag = f"SVJ{i}"
        assert f"){tag}\"" not in text
        names.append(f'"{h}"')
        texts.append(f'R"{tag}({text}){tag}"')
    parts.append(f"static constexpr int kJitHeaderCount = {len(JIT_HEADERS)};\n")
    parts.append("static const char* const kJitHeaderNames[] = {" + ", ".join(names) + "};\n")
    parts.append("static const char* const kJitHeaders[] = {\n" + ",\n".join(texts) + "};\n")
    content = "".join(parts)
    if not os.path.exists(path) or open(path).read() != content:
        with open(path, "w") as f:
            f.write(content)
    return path


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, src + ".o")
    path = os.path.join(CSRC, src)
    deps = [path] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    deps.append(os.path.join(INCLUDE, "sv.h"))
    deps.append(os.path.join(BUILD, "jit_embed.inc"))
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in deps):
        return obj
    cmd = [NVCC] + _flags() + ["-c", path, "-o", obj]
    if src.endswith(".cu") and verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        sys.stderr.write(r.stdout + r.stderr)
    return obj


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "arch.txt")
    arch = platform.machine()
    if not os.path.exists(stamp) or open(stamp).read().strip() != arch:
        force = True  # objects from another host architecture are unusable here
    if force:
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
        if os.path.exists(OUT):
            os.remove(OUT)
        with open(stamp, "w") as f:
            f.write(arch + "\n")
    _write_jit_embed()
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    if (not force and os.path.exists(OUT)
            and os.path.getmtime(OUT) >= max(os.path.getmtime(o) for o in objs)):
        return OUT
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
