"""Writes tests/golden/full_size_counts.txt: expected values for the full-size workloads.

Every value comes from the CPU oracle (oracle/) on inputs from synth/ only; nothing here
touches the CUDA path. Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_size_counts.txt")


def main():
    oracle.set_threads(0)
    rows = []
    t0 = time.time()
    c = synth.cfg1()
    rows.append(("cfg1_n4096_r2_16", oracle.count_i32(c["x"], c["y"], c["z"], 16), ""))
    for n in (262144, 262145):
        c = synth.cfg2(n)
        rows.append((f"cfg2_n{n}_r2_9", oracle.count_i32(c["x"], c["y"], c["z"], 9), ""))
        s = synth.cfg2(n, same_cell=True)
        v = oracle.count_i32(s["x"], s["y"], s["z"], 0)
        assert v == oracle.count_colls(s["x"], s["y"], s["z"])   # Algorithm 1 cross-check
        rows.append((f"cfg2_samecell_n{n}_r2_0", v, ""))
        p = synth.cfg2_planted(n)
        rows.append((f"cfg2_planted_n{n}_r2_9", oracle.count_i32(p["x"], p["y"], p["z"], 9), ""))
    c = synth.cfg3()
    cnt, sm = oracle.count_f32(c["x"], c["y"], c["z"], c["r"])
    rows.append(("cfg3_n131072_f32", cnt, repr(sm)))
    with open(OUT, "w") as f:
        f.write("# Expected results of the full-size workloads, written by tests/golden/make_golden.py\n")
        f.write("# from the CPU oracle (standard pairwise loop of Section 4) on synth/ inputs.\n")
        f.write("# name count [fp64_sum]\n")
        for name, v, extra in rows:
            f.write(f"{name} {v} {extra}".rstrip() + "\n")
    print(open(OUT).read(), f"{time.time() - t0:.1f}s")


if __name__ == "__main__":
    main()
