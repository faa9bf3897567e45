"""Builds and runs the arithmetic throughput probe (qb_peak_probe.cu) on the
current GPU and prints its measurements."""
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))

if __name__ == "__main__":
    exe = os.path.join(tempfile.mkdtemp(), "qb_peak_probe")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                           os.path.join(HERE, "qb_peak_probe.cu")])
    sys.exit(subprocess.call([exe]))
