"""Reconstruction error and bit-rate accounting.

Test infrastructure (see ``oracle/__init__``).

* ``nmse`` - sum ||a~ - a||^2 over all vertex-frames divided by
  sum_f sum_i ||a_{f,i} - abar_f||^2 (abar_f the centroid of frame f).
  The paper reports NMSVE [its ref. 4], which it does not define; NMSE of
  this form is the error measure the codec is checked with.  numpy's
  pairwise summation is used on contiguous arrays.
* ``rates`` - Eq. 13: bits per vertex per frame of the coefficients (q),
  the anchors (q_a), the dictionary (q_d) and their total (q_s), with F
  frames (the paper's k), n_b blocks of k_f = F / n_b frames.
  q   = bits_coeff * n * k / (n * F)   for k retained rows of the n-column
        coefficient matrix (Eq. 13 prints "bits * n * k / (n * k)" with the
        paper's k for frames; counting the k_l coded rows is the reading
        under which it is not identically ``bits``)
  q_a = bits_anchor * n_c * F / (n * F)
  q_d = bits_dict * n_b^2 * k_f * k_f / (n * F)   (a full F x F dictionary
        per the paper; ``dict_cols`` lets the caller count only the k
        columns the codec transmits)

Pinned by Table I: q_d = 0.2799 (Handstand, n = 10002, F = 175),
0.2808 (Samba, n = 9971), q_a = 0.1600 (Handstand, n_c = 1% of n), and
the q_s column sums (tests/golden/table1_rates.txt).
"""

import numpy as np


def nmse(a, a_rec):
    a = np.asarray(a, dtype=np.float64)
    a_rec = np.asarray(a_rec, dtype=np.float64)
    err = np.sum((a_rec - a) ** 2)
    centred = a - a.mean(axis=1, keepdims=True)
    return float(err / np.sum(centred ** 2))


def rates(n, F, k, n_anchors, coeff_bits, anchor_bits, dict_bits, n_b=1, dict_cols=None):
    k_f = F / n_b
    q = coeff_bits * n * k / (n * F)
    q_a = anchor_bits * n_anchors * F / (n * F)
    if dict_cols is None:
        q_d = dict_bits * n_b ** 2 * k_f * k_f / (n * F)
    else:
        q_d = dict_bits * n_b * k_f * dict_cols / (n * F)
    return {"q": q, "q_a": q_a, "q_d": q_d, "q_s": q + q_a + q_d}
