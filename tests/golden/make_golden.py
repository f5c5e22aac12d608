"""Write tests/golden/golden.json: fingerprints of ORACLE outputs on the
full-size seeded workloads, for GPU parity tests at sizes the oracle cannot
recompute inside a test run.

Calls only the CPU oracle (oracle/) and the seeded input generators (synth.py);
nothing here touches the CUDA path.  Each entry stores the SHA-256 of the
oracle's output (little-endian uint64, C order), its shape, and a few sampled
values.  Run once (about 25 minutes on 8 cores):

    python tests/golden/make_golden.py [name ...]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "golden.json")


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a.astype(np.uint64)).tobytes()).hexdigest()


def samples(a: np.ndarray, n=8):
    flat = a.reshape(-1)
    idx = np.linspace(0, flat.size - 1, n).astype(np.int64)
    return [[int(i), int(flat[i])] for i in idx]


def product(name, ntt_prime):
    W = synth.product_c2(0, ntt_prime=ntt_prime)
    C = oracle.pmat_mul(W["p"], W["A"], W["B"])
    return {"what": "pmat_mul, 32x32 . 32x32, length 4096, seed 0", "p": W["p"], "shape": list(C.shape),
            "sha256": digest(C), "samples": samples(C), "oracle": "orc_pmat_slice (product as the convolution sum)"}


def pmbasis():
    W = synth.pmbasis_c3(0)
    P, rd = oracle.mbasis(W["p"], W["F"], W["d"], W["shift"])
    return {"what": "M-Basis (Algorithm 2) = PM-Basis (Algorithm 3), F 32x16, order 8192, shift 0, seed 0",
            "p": W["p"], "shape": list(P.shape), "sha256": digest(P), "samples": samples(P),
            "rdeg": [int(v) for v in rd], "oracle": "orc_mbasis"}


def resultant():
    W = synth.resultant_c5(0, nprimes=1)
    R = oracle.bivariate_resultant(W["primes"][0], W["f"][0], W["g"][0])
    return {"what": "Res_y(f, g), f, g dense with deg_x = deg_y = 150, seed 0", "p": W["primes"][0],
            "shape": list(R.shape), "sha256": digest(R), "samples": samples(R),
            "oracle": "orc_bivariate_resultant (evaluate / Euclid / Newton interpolation)"}


def resultant_16():
    """The 16-prime batch: the same integer coefficients reduced modulo 16 random 60-bit primes,
    one oracle resultant per prime."""
    W = synth.resultant_c5(0, nprimes=16)
    shas, samp = [], []
    for i, p in enumerate(W["primes"]):
        R = oracle.bivariate_resultant(p, W["f"][i], W["g"][i])
        shas.append(digest(R))
        samp.append(samples(R, 4))
    return {"what": "Res_y(f, g) modulo each of 16 primes, f, g dense with deg_x = deg_y = 150, seed 0",
            "primes": [int(p) for p in W["primes"]], "shape": [16, 45001], "sha256": shas, "samples": samp,
            "oracle": "orc_bivariate_resultant (evaluate / Euclid / Newton interpolation), once per prime"}


JOBS = {"product_32x32_p60": lambda: product("p60", False),
        "product_32x32_p998": lambda: product("p998", True),
        "pmbasis_32x16_d8192": pmbasis,
        "resultant_150": resultant,
        "resultant_150_16primes": resultant_16}


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for nm in names or list(JOBS):
        t0 = time.time()
        data[nm] = JOBS[nm]()
        data[nm]["oracle_seconds"] = round(time.time() - t0, 1)
        data[nm]["oracle_threads"] = oracle.max_threads()
        json.dump(data, open(OUT, "w"), indent=1)
        print(nm, data[nm]["oracle_seconds"], "s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
