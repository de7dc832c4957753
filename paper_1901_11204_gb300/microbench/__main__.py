"""Builds and runs the TMEM read / tensor-core MMA rate microbenchmark (tmem_mma_rates.cu)
on the current GPU; prints its JSON line. The rates are the hardware bounds that bench.py
reports beside the tensor-core pair kernel's measured rate."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def build() -> str:
    """Compiles the microbenchmark for sm_103a (the package's nvcc and architecture flags)
    and returns the executable's path."""
    sys.path.insert(0, os.path.dirname(HERE))
    import builder  # noqa: E402  (the package's nvcc location and flags)
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    exe = os.path.join(out, "tmem_mma_rates")
    cmd = [builder._nvcc(), *builder.ARCH, "-O3", "-std=c++17", "--expt-relaxed-constexpr",
           "-I" + os.path.join(ROOT, "include"), os.path.join(HERE, "tmem_mma_rates.cu"), "-o", exe]
    subprocess.run(cmd, check=True)
    return exe


def main() -> int:
    return subprocess.run([build()]).returncode


if __name__ == "__main__":
    sys.exit(main())
