"""Write the committed table bytes of the benchmark's large scalar.

large_n50_g2000_t80_seed0.zxps: the seeded large workload (n = 50 qubits,
2000 gates with 80 T gates, seed 0, its random output bitstring) reduced by
the library's compiler with its default split (a version-2 table: outer and
inner parameters).  The CPU oracle times its sum from these bytes in the
benchmark's reference arm, so that arm does not load the library; the test
suite checks that a fresh compile still gives the same bytes.

    python zxp_inputs/tables/make_tables.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

LARGE = os.path.join(HERE, "large_n50_g2000_t80_seed0.zxps")


def large_blob() -> bytes:
    import paper_2403_06777_gb300 as Z
    import zxp_inputs as zi
    w = zi.workload_large(0)
    return Z.zxp_scalar_to_tables(Z.zxp_compile(w.gates, w.n, w.out_bits))


if __name__ == "__main__":
    with open(LARGE, "wb") as f:
        f.write(large_blob())
    print(LARGE)
