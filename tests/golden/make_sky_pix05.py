"""Write the FP64 oracle's results for the 0.5-degree diffuse-sky member.

The oracle's left-looking factorization of this member (19,600 sky columns,
largest front about 13,500 rows) takes about an hour on one core, too long
for a test, so its results are stored: x for b, and the variances of the sky
columns, with a fingerprint of the generated matrix.  Inputs come from the
seeded generator; every stored value comes from oracle/ alone.

    python tests/golden/make_sky_pix05.py      # writes sky_pix05_oracle.npz here
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from spigen import SKY_PIX05, generate  # noqa: E402

OUT = os.path.join(HERE, "sky_pix05_oracle.npz")


def fingerprint(pb) -> np.ndarray:
    """sum of N's stored values, sum of b, and N r for a fixed r (first 64 entries)."""
    r = np.random.default_rng(123).uniform(-1.0, 1.0, pb.n)
    Nr = pb.full_matrix() @ r
    return np.concatenate([[pb.values.sum(), pb.b.sum()], Nr[:64]])


def main():
    t0 = time.time()
    pb = generate(SKY_PIX05)
    t1 = time.time()
    f = oracle.OracleFactor.from_problem(pb)
    t2 = time.time()
    x = f.solve(pb.b)
    var_sky = f.inv_diag(pb.sky_columns)
    t3 = time.time()
    np.savez_compressed(OUT, x=x, var_sky=var_sky, sky_columns=pb.sky_columns, n=pb.n, nnz=pb.nnz,
                        fingerprint=fingerprint(pb),
                        seconds=np.array([t1 - t0, t2 - t1, t3 - t2]))
    print(f"n={pb.n} nnz={pb.nnz} sky={pb.n_sky}: generate {t1 - t0:.1f} s, oracle factor {t2 - t1:.1f} s, "
          f"solve + sky variances {t3 - t2:.1f} s -> {OUT}")


if __name__ == "__main__":
    main()
