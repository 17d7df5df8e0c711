"""Writes batched_residuals.json: for each of the 64 obstacles of the batched
workload (64 seeded bodies, N ~ U[60, 360], P in {32, 64, 120, 180, 240},
k ~ U[1, 30], Neumann or transmission), the oracle's least-squares residual
||A c - fhat|| / ||fhat|| on the 4 plane waves the batched parity test uses
(seed 500 + index), and the oracle's own sensitivity: e_bd between its
solution and its solution with every modal matrix perturbed by u max|A|
complex Gaussian noise (seed 123 + index). Calls only the oracle.

An obstacle with residual > 1e-6 is unresolved: N, P and k are drawn
independently, so the discretisation cannot represent the field, and the
least-squares solution is not determined to 1e-10 by the data.

Run: python tests/golden/batched_residuals.py   (about half an hour on 8 cores)
"""
import dataclasses
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import synth  # noqa: E402


def residual_and_sensitivity(i, ob):
    coll, src, srcx = O.geometry(ob)
    ob = dataclasses.replace(ob, q=O.choose_q(ob, coll, src, srcx))
    A, fac = O.factor_operator(ob, coll, src, srcx)
    dirs = synth.plane_wave_directions(4, 500 + i)
    fh = O.rhs_modes(O.incident_samples(ob, coll, dirs))
    c = O.solve_modes(ob, fac, fh)
    P = ob.P
    red = lambda idx: idx if idx <= P // 2 else P - idx
    res = math.sqrt(sum(np.linalg.norm(A[red(idx)] @ c[:, idx].T - fh[:, idx].T) ** 2
                        for idx in range(P))) / np.linalg.norm(fh)
    rng = np.random.default_rng(123 + i)
    u = np.finfo(float).eps / 2
    num = 0.0
    cols = A.shape[2]
    for idx in range(P):
        n = red(idx)
        noise = rng.standard_normal(A[n].shape) + 1j * rng.standard_normal(A[n].shape)
        QR, tau = O.householder_qr(A[n] + u * np.abs(A[n]).max() * noise / math.sqrt(2))
        y = O.apply_qh(QR, tau, fh[:, idx, :].T)[:cols]
        cp = O.back_substitute(np.triu(QR[:cols, :cols]), y)
        num += np.linalg.norm(A[n] @ (c[:, idx].T - cp)) ** 2
    return {"index": i, "N": ob.N, "M": ob.M, "P": ob.P, "q": ob.q, "k": ob.k, "bc": ob.bc,
            "residual": res, "sensitivity": math.sqrt(num) / np.linalg.norm(fh)}


def main():
    out = os.path.join(HERE, "batched_residuals.json")
    done = json.load(open(out)) if os.path.exists(out) else {}
    wl = synth.config_batched()
    for i, ob in enumerate(wl.obstacles):
        if str(i) in done:
            continue
        done[str(i)] = residual_and_sensitivity(i, ob)
        print(i, done[str(i)], flush=True)
        json.dump(done, open(out, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
