"""Writes tests/golden/scale_oracle.txt: the CPU oracle's Z(q) and V_K(t(q)) for the
64-knot grid-walk workload (L = 40, seeds 1..64, 100..400 crossings, random over/under)
at q = 2, 3, 5 -- every (knot, q) pair whose min-fill spin elimination keeps every
summed-out factor within q^(w-1) <= 5^12 entries (w spins in the bucket, the one summed
out included): the six q = 5 pairs with 14 or 15 spins per bucket are left out.

Z is the plain spin sum of Sec. II summed out one spin at a time (`oracle.z_complex`,
complex128 with a power-of-two exponent per factor; order from `oracle.order`), V = A(q) Z
(Eq. JonesPotts, `oracle.jones_from_z`).  Only `knotgen` (inputs) and `oracle` are used.
Values are stored as hexadecimal floats (exact).  Run: python tests/golden/make_scale_oracle.py
"""
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "scale_oracle.txt")
MAX_ENTRIES = 5 ** 12
QS = (2, 3, 5)


def fits(q, w):
    return q ** (w - 1) <= MAX_ENTRIES


def one(job):
    sys.path.insert(0, ROOT)
    import knotgen as kg
    import oracle
    from oracle.order import min_fill_order
    seed, q = job
    gk = kg.random_grid_knot(40, seed, True, 100, 400)
    g = oracle.tait_graph(gk.pd, outer=gk.outer)
    order, w = min_fill_order(g.n_v, g.edges, q, seed=0, restarts=16)
    if not fits(q, w):
        return seed, q, w, None, None
    z = oracle.z_complex(g.n_v, g.edges, q, order=order, sum_inside=True)
    v = oracle.jones_from_z(z, g, q)
    return seed, q, w, z, v


def main():
    sys.path.insert(0, ROOT)
    import oracle.order  # noqa: F401  (fail early if the package is missing)
    jobs = [(s, q) for s in range(1, 65) for q in QS]
    procs = int(os.environ.get("ORACLE_PROCS", "4"))
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"      # one thread per worker process
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(one, jobs, chunksize=1)
    with open(OUT, "w") as f:
        f.write("# CPU oracle: Z(q) (Sec. II spin sum) and V = A(q) Z (Eq. JonesPotts) of the\n"
                "# L=40 grid-walk workload (seeds 1..64, 100..400 crossings, random over/under);\n"
                "# written by tests/golden/make_scale_oracle.py.  Columns: seed q width\n"
                "# Z.re Z.im Z.exp2 V.re V.im V.exp2 (value = (re + i im) 2^exp2, hex floats);\n"
                "# pairs whose buckets exceed 5^12 entries are listed with '-' values\n")
        for seed, q, w, z, v in res:
            if z is None:
                f.write(f"{seed} {q} {w} - - - - - -\n")
            else:
                f.write(f"{seed} {q} {w} {z.m.real.hex()} {z.m.imag.hex()} {z.e} "
                        f"{v.m.real.hex()} {v.m.imag.hex()} {v.e}\n")
    print(f"wrote {OUT}: {sum(z is not None for _, _, _, z, _ in res)} of {len(res)} pairs")


if __name__ == "__main__":
    main()
