"""Write the oracle reference solutions used by the GPU tests (calls only oracle/ and synthetic/).

    python tests/golden/make_references.py [c3|meg_faust]   (both when no name is given)

c3_reference.npz: for 20 signals of the c3 batch (2048 x 8192, seed 0) the Lasso minimiser at
lambda = ratio * lambda_max, computed by the FP64 oracle (FISTA + GAP Safe, then the KKT-verified
support system), stored sparsely (support, values), with lambda_max and lambda.
meg_faust_reference.npz: the same for sampled signals of the source-localisation stand-in
(204 x 8193 dense A, 50 signals, lambda = 0.1 lambda_max, seed 0).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synthetic as S                      # noqa: E402
from oracle import lasso as OL             # noqa: E402
from oracle import solvers as OS           # noqa: E402

# c3 signals compared element by element: the first ones, the four smallest and four largest
# lambda / lambda_max, the three densest and two sparsest x0, one in the middle and the ragged
# end of the batch (chosen from the generator's draws for seed 0)
C3_SIGNALS = (0, 1, 2, 15, 315, 1771, 2048, 2084, 2187, 2284, 2298, 3235, 3328, 3513, 3610, 3670, 3810,
              4093, 4094, 4095)
MEG_SIGNALS = (0, 23, 49)


def minimiser(A, y, lam):
    for tol in (1e-9, 1e-11, 1e-13):
        r = OS.fista_gap_safe(A, y, lam, tol, max_iter=400000)
        x, ok = OS.kkt_polish(A, y, lam, r.x)
        if ok:
            return x
    raise RuntimeError("oracle did not identify the support")


def sampled_reference(path, w, signals):
    out = {}
    for b in signals:
        y = w.Y[b]
        lm = OL.lambda_max(w.A.T @ y)
        lam = float(w.lam_ratio[b]) * lm
        x = minimiser(w.A, y, lam)
        S_ = np.flatnonzero(x)
        out[f"s{b}_idx"] = S_.astype(np.int32)
        out[f"s{b}_val"] = x[S_]
        out[f"s{b}_lmax"] = np.array(lm)
        out[f"s{b}_lam"] = np.array(lam)
        print(b, "support", S_.size, "lambda/lambda_max", w.lam_ratio[b])
    out["signals"] = np.array(signals)
    np.savez_compressed(path, **out)


if __name__ == "__main__":
    which = sys.argv[1:] or ["c3", "meg_faust"]
    if "c3" in which:
        sampled_reference(os.path.join(HERE, "c3_reference.npz"), S.c3(n_signals=4096), C3_SIGNALS)
    if "meg_faust" in which:
        sampled_reference(os.path.join(HERE, "meg_faust_reference.npz"), S.meg_faust(n_signals=50), MEG_SIGNALS)
