"""Build and run the instruction issue-rate probe (probe/pipes.cu) on the
current GPU; prints one JSON line per instruction kind.

    python -m paper_0804_3643_gb300.peak

Under ncu, with --metrics sm__inst_executed_pipe_alu.sum,
sm__inst_executed_pipe_fmaheavy.sum,smsp__inst_executed.sum, it shows on which
pipe each kind issues: integer maxima on the ALU pipe, int16x2 adds and IMAD
on the FMA-heavy pipe, each about 64 lanes per clock per SM.  The integer
rooflines bench.py reports (stage 2 and stage 3.1) rest on that split.
"""
import os
import subprocess
import sys

from .build import ARCH, nvcc

HERE = os.path.dirname(os.path.abspath(__file__))


def main() -> int:
    src = os.path.join(HERE, "probe", "pipes.cu")
    exe = os.path.join(HERE, "probe", "pipes")
    subprocess.check_call([nvcc()] + ARCH + ["-O3", "-o", exe, src])
    return subprocess.call([exe])


if __name__ == "__main__":
    sys.exit(main())
