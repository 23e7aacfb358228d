"""Compile the CPU oracle (test infrastructure) into oracle/liboracle.so.

gcc, C99, -O2 -ffp-contract=off (no fused multiply-add), single-threaded.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbdps_oracle.c")
OUT = os.path.join(HERE, "liboracle.so")


def build_to(src: str, out: str, quiet: bool = False) -> str:
    """Compile ``src`` into the shared library ``out`` with the oracle's flags
    (``quiet``: compiler messages are dropped unless the compile fails)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC",
           "-shared", "-Wall", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True, capture_output=quiet)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    return build_to(SRC, OUT)


if __name__ == "__main__":
    print(build(force=True))
