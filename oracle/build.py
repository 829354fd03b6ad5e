"""Build the oracle shared library (test infrastructure only).

Compiles the plain C sources of this directory with gcc into
``liboracle.so`` next to them.  No fast-math, no target-specific flags: the
same source gives the same results on x86-64 and AArch64 (no FMA
contraction: every product and sum is rounded on its own).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["philox.c", "rules.c", "obs.c", "belief.c", "drivers.c", "search.c", "policy.c"]
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False, out: str = LIB, extra=()) -> str:
    """Build the library at `out` (default: liboracle.so here) with the
    standard flags plus `extra` (the tests build a sanitizer variant into a
    temporary directory this way)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "oracle.h")]
    if not force and os.path.exists(out):
        t = os.path.getmtime(out)
        if all(os.path.getmtime(d) <= t for d in deps):
            return out
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra", "-Wno-unused-parameter",
           "-fno-fast-math", "-ffp-contract=off"] + list(extra) + ["-o", tmp] + srcs
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
