"""Build the CUDA library ``_lib/libetd_gb300.so`` (sm_103a) in-tree.

One translation unit per (dtype, axis length) instantiation of the pass kernel is generated under
``_build/gen`` and compiled in parallel with nvcc; the host executor (``csrc/etd_api.cu``) and the
kernel registry are linked in with the static CUDA runtime. ptxas register/spill reports go to
``_build/ptxas.log``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
GEN = os.path.join(BUILD, "gen")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libetd_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
LENGTHS = [4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 6, 12, 24, 48, 96, 192, 384, 768, 1536]
TYPES = {"f32": "float", "f64": "double"}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags():
    return ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
            "-Xptxas", "-v", f"-I{CSRC}", f"-I{INCLUDE}"]


def _write_if_changed(path: str, text: str) -> None:
    if os.path.exists(path) and open(path).read() == text:
        return
    with open(path, "w") as fh:
        fh.write(text)


def generate() -> list:
    os.makedirs(GEN, exist_ok=True)
    srcs = []
    decls, rows = [], []
    for tk, tn in TYPES.items():
        # transform variants (enum Variant of dst_engine.cuh): 1 odd extension (FP32 only),
        # 0 half-length recurrence, 2 Hartley (periodic axes)
        for v, o in ((("odd", 1), ("rec", 0), ("hart", 2)) if tk == "f32" else (("rec", 0), ("hart", 2))):
            for n in LENGTHS:
                name = f"kinfo_{tk}_{v}_{n}"
                path = os.path.join(GEN, f"inst_{tk}_{v}_{n}.cu")
                _write_if_changed(path, (
                    '#include "pass_kernel.cuh"\n'
                    "namespace etd {\n"
                    f"template __global__ void pass_kernel<{tn}, {n}, {o}>(const PassArgs<{tn}>);\n"
                    f"template __global__ void pass_kernel_batched<{tn}, {n}, {o}>(const PassArgs<{tn}>*, const int2*, {tn}* const*);\n"
                    f"KernelInfo {name}() {{ return kernel_info<{tn}, {n}, {o}>(); }}\n"
                    "}  // namespace etd\n"))
                srcs.append(path)
                decls.append(f"KernelInfo {name}();")
                rows.append(f"    {name}(),")
    reg = os.path.join(GEN, "registry.cu")
    _write_if_changed(reg, (
        '#include "pass_kernel.cuh"\n'
        "namespace etd {\n" + "\n".join(decls) + "\n"
        "const KernelInfo* find_pass_kernel(int elem, int N, int variant) {\n"
        "  static const KernelInfo table[] = {\n" + "\n".join(rows) + "\n  };\n"
        "  for (const KernelInfo& k : table)\n"
        "    if (k.elem == elem && k.N == N && k.odd == variant) return &k;\n"
        "  return nullptr;\n"
        "}\n"
        "}  // namespace etd\n"))
    srcs.append(reg)
    srcs.append(os.path.join(CSRC, "etd_api.cu"))
    srcs.append(os.path.join(CSRC, "monitor_noalloc.cu"))
    srcs.append(os.path.join(CSRC, "gemm_inst.cu"))
    srcs.append(os.path.join(CSRC, "split_inst.cu"))
    srcs.append(os.path.join(CSRC, "sno.cu"))
    return srcs


def _compile(src: str) -> tuple:
    obj = os.path.join(BUILD, "obj", os.path.basename(src).replace(".cu", ".o"))
    os.makedirs(os.path.dirname(obj), exist_ok=True)
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "etd.h"), os.path.join(INCLUDE, "etd_sno.h")]
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in deps):
        return obj, ""
    cmd = [nvcc(), *_flags(), "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(jobs: int | None = None, verbose: bool = False) -> str:
    srcs = generate()
    jobs = jobs or max(1, min(len(srcs), os.cpu_count() or 4))
    logs = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = []
        for obj, log in ex.map(_compile, srcs):
            objs.append(obj)
            if log:
                logs.append(log)
    if logs:
        with open(os.path.join(BUILD, "ptxas.log"), "w") as fh:
            fh.write("\n".join(logs))
    os.makedirs(LIBDIR, exist_ok=True)
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared", *ARCH, "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build(verbose=True, jobs=int(sys.argv[1]) if len(sys.argv) > 1 else None)
