"""Compile libhh (the CUDA sources under csrc/) in-tree for sm_103a with nvcc.

The translation units are compiled in parallel as relocatable device code and
linked into one shared library: the host/kernel unit hh_host.cu, the
surrogate network hh_cnn.cu, the compiled-shape field kernels hh_ct_inst.cu
once per kernel (plane passes in four shape groups, and the column pass),
and the two-pass transform table hh_fft2_inst.cu once per (precision,
direction).
"""

import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libhh.so")
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")

# (source, object name, extra flags)
UNITS = [("hh_host.cu", "hh_host.o", []), ("hh_cnn.cu", "hh_cnn.o", [])] + [
    ("hh_ct_inst.cu", "hh_ct_%d.o" % part, ["-DHH_CT_PART=%d" % part]) for part in range(9)] + [
    ("hh_fft2_inst.cu", "hh_fft2_%s.o" % name, ["-DHH_FFT2_T=%s" % t, "-DHH_FFT2_INV=%d" % inv,
                                                  "-DHH_FFT2_NAME=fft2_%s" % name])
    for name, t, inv in (("f32_fwd", "float", 0), ("f32_inv", "float", 1), ("f64_fwd", "double", 0),
                         ("f64_inv", "double", 1))]
DEPS = [os.path.join(CSRC, f) for f in ("hh_host.cu", "hh_cnn.cu", "hh_fft2_inst.cu", "hh_device.cuh", "hh_post.cuh",
                                        "hh_fused.cuh", "hh_plane_ct.cuh", "hh_ct_inst.cu",
                                        "hh_fftcore.cuh", "hh_fft2.cuh", "hh_ctmath.h", "hh_internal.h")] + [
    os.path.join(ROOT, "include", "hh.h"), os.path.abspath(__file__)]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Relocatable device code: a kernel's register count after linking is the
# largest over everything it calls, so one cap for every unit keeps the
# transform functions from setting the occupancy of the field kernels
# (64 registers: four 256-thread blocks per SM, matching the launch bounds).
MAX_REGS = 64
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-rdc=true", "-Xcompiler", "-fPIC"]


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
    return res.stdout + res.stderr


def build(force: bool = False, verbose: bool = False, extra=(), max_regs: int = MAX_REGS, lib: str = LIB,
          build_dir: str = BUILD_DIR) -> str:
    """Build libhh.so next to this file (or at `lib`); returns its path."""
    if not force and lib == LIB and up_to_date():
        return LIB
    os.makedirs(build_dir, exist_ok=True)
    nvcc = nvcc_path()
    inc = "-I" + os.path.join(ROOT, "include")
    cmds, objs = [], []
    for src, obj, flags in UNITS:
        o = os.path.join(build_dir, obj)
        objs.append(o)
        cmds.append([nvcc, *NVCC_FLAGS, "-maxrregcount=%d" % max_regs, *extra, *flags, inc, "-c", "-o", o,
                     os.path.join(CSRC, src)])
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        outs = [f.result() for f in [ex.submit(_run, c, verbose) for c in cmds]]
    if verbose:
        for out in outs:
            print(out)
    tmp = lib + ".tmp"
    _run([nvcc, *ARCH, "-rdc=true", "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs], verbose)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
