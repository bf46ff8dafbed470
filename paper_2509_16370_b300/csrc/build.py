"""Build the CUDA library librlqr.so in-tree for sm_103a with nvcc.

Usage: python -m paper_2509_16370_b300.csrc.build [--force]
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.dirname(HERE)
OUT_DIR = os.path.join(PKG, "_lib")
OUT = os.path.join(OUT_DIR, "librlqr.so")
SOURCES = ["rlqr_api.cu", "launch_fp32.cu", "launch_fp64.cu", "scan_fp32.cu", "scan_fp64.cu",
           "shard.cu", "pipes.cu", "ipm.cu", "mlp.cu", "diag.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
         "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-Xptxas", "-v"]


def _stale():
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    deps = [os.path.join(HERE, d) for d in os.listdir(HERE) if d.endswith((".cu", ".cuh"))]
    deps += [os.path.join(os.path.dirname(PKG), "include", h) for h in ("rlqr.h", "rlqr_ipm.h", "rlqr_mlp.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the translation units in parallel, then link librlqr.so."""
    if not force and not _stale():
        return OUT
    os.makedirs(OUT_DIR, exist_ok=True)
    objs = [os.path.join(OUT_DIR, os.path.splitext(s)[0] + f".{os.getpid()}.o") for s in SOURCES]
    cmds = [[NVCC] + FLAGS + ["-c", "-o", o, os.path.join(HERE, s)]
            for s, o in zip(SOURCES, objs)]
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for c in cmds]
    outs = [p.communicate() for p in procs]
    log = os.path.join(OUT_DIR, "build.log")
    with open(log, "w") as f:
        for c, (o, e) in zip(cmds, outs):
            f.write(" ".join(c) + "\n" + o + e)
    failed = [i for i, p in enumerate(procs) if p.returncode != 0]
    if failed:
        for i in failed:
            sys.stderr.write(outs[i][1][-6000:])
        raise RuntimeError(f"nvcc failed (see {log})")
    tmp = OUT + f".tmp{os.getpid()}"
    link = [NVCC, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp] + objs
    res = subprocess.run(link, capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if res.returncode != 0:
        sys.stderr.write(res.stderr[-4000:])
        raise RuntimeError("nvcc link failed")
    if verbose:
        sys.stderr.write("".join(e for _, e in outs))
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
