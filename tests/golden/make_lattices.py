"""Write tests/golden/lattices.json: CBC generating vectors from the oracle only.

For every prime the tests and parity checks use (the lattice-size ladder, the
64-entry batch table, 10007 and the 65537 pilot size) this runs the oracle's
fast component-by-component search with product weights gamma_i = 1/i^2 up to
d = 10.  A CBC vector for d dimensions is the first d entries of the longer
one, so one table serves every dimension <= 10.

    python tests/golden/make_lattices.py [--max-n N]
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle.cbc import cbc_fast  # noqa: E402
from paper_1811_11722_gb300 import inputs as I  # noqa: E402

DMAX = 10


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--max-n", type=int, default=1 << 62)
    ap.add_argument("--out", default=os.path.join(HERE, "lattices.json"))
    args = ap.parse_args()
    primes = sorted(set([I.N_C1, I.N_PILOT] + I.ladder_primes() + I.batch_prime_table()))
    primes = [p for p in primes if p <= args.max_n]
    table = {}
    if os.path.exists(args.out):
        table = json.load(open(args.out)).get("g", {})
    gamma = I.product_weights(DMAX)
    for n in primes:
        if str(n) in table:
            continue
        t = time.time()
        g = cbc_fast(DMAX, n, gamma)
        table[str(n)] = [int(v) for v in g]
        print(f"n={n} g={table[str(n)]} {time.time() - t:.1f}s", flush=True)
        json.dump({"criterion": "shift-averaged worst-case error, unanchored weighted Sobolev space, "
                                "product weights gamma_i = 1/i^2, CBC with g_1 = 1 (oracle/cbc.py)",
                   "dmax": DMAX, "g": dict(sorted(table.items(), key=lambda kv: int(kv[0])))},
                  open(args.out, "w"), indent=0)


if __name__ == "__main__":
    main()
