"""Measure the issue rates that the ALU rooflines are quoted against.

Compiles ``csrc/alu_probe.cu`` (sm_103a) into ``_build/alu_probe`` and runs it
on the current GPU.  Prints one JSON object with results per clock per SM for
packed FP32 FMA (FFMA2, two results per instruction), scalar FP32 FMA, the MUFU
approximations lg2/rcp/ex2/rsqrt/sin and FP64 FMA, plus the SM count.

    python -m paper_2111_01083_gb300.alu_peaks > profiles/alu_peaks.json
"""
import json
import os
import subprocess
import sys

from .build import ARCH, OBJ, CSRC, _nvcc


def measure():
    os.makedirs(OBJ, exist_ok=True)
    exe = os.path.join(OBJ, "alu_probe")
    src = os.path.join(CSRC, "alu_probe.cu")
    if not os.path.exists(exe) or os.path.getmtime(exe) < os.path.getmtime(src):
        r = subprocess.run([_nvcc(), *ARCH, "-O3", "-std=c++17", src, "-o", exe], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for alu_probe.cu:\n{r.stderr}")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    if r.returncode != 0:
        raise RuntimeError(f"alu_probe failed ({r.returncode}): {r.stdout} {r.stderr}")
    return json.loads(r.stdout.strip().splitlines()[-1])


if __name__ == "__main__":
    json.dump(measure(), sys.stdout)
    sys.stdout.write("\n")
