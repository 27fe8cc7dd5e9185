"""Writes const_2layer_moments.json: exact moments of the outflow Q_l for the
two-layer piecewise-constant model (Sec. 2 Ex. 1 with one random horizontal
interface, Sec. 3.4 Model Problem 2).

With horizontal layers the discrete outflow is the arithmetic mean of the row
permeabilities, so Q_l = k_2 + (k_1 - k_2) w_l where w_l = n_l(eta)/m_l is the
fraction of row centres below eta ~ U(a, b), n_l(eta) = ceil(m_l eta - 1/2),
and k_t = exp(Z_t), Z_t ~ N(0, 1) independent: E[k] = e^(1/2), E[k^2] = e^2,
E[k_1 k_2] = e.  The expectations over eta are exact sums over the intervals
on which the step functions w_l are constant.  Uses only the closed form (no
solver, no sampler)."""
import json
import math
import os
from fractions import Fraction


def eta_moments(ms, a, b):
    """Exact E[f(w_{m_1}, w_{m_2}, ...)] helpers: list of (prob, [w per m])."""
    pts = {Fraction(a), Fraction(b)}
    for m in ms:
        for j in range(m):
            y = Fraction(2 * j + 1, 2 * m)
            if Fraction(a) < y < Fraction(b):
                pts.add(y)
    pts = sorted(pts)
    out = []
    for lo, hi in zip(pts[:-1], pts[1:]):
        mid = (lo + hi) / 2
        ws = [Fraction(math.ceil(m * mid - Fraction(1, 2)), m) for m in ms]
        out.append(((hi - lo) / (Fraction(b) - Fraction(a)), ws))
    return out


def main():
    e = math.e
    ms = [8, 16, 32]
    a, b = Fraction(3, 10), Fraction(7, 10)
    pieces = eta_moments(ms, a, b)
    res = {"source": "closed form of Sec. 2 Ex. 1 with Sec. 3.4 Model Problem 2; "
                     "eta ~ U(0.3, 0.7), Z ~ N(0, 1)",
           "E_Q": math.exp(0.5), "V_Q": {}, "V_Y": {}}
    for li, m in enumerate(ms):
        Ew = float(sum(p * w[li] for p, w in pieces))
        Ew2 = float(sum(p * w[li] ** 2 for p, w in pieces))
        EQ2 = e * e * (1 - 2 * Ew + 2 * Ew2) + 2 * e * (Ew - Ew2)
        res["V_Q"][str(m)] = EQ2 - e
    for li in (1, 2):
        Ed2 = float(sum(p * (w[li] - w[li - 1]) ** 2 for p, w in pieces))
        res["V_Y"]["%d_%d" % (ms[li], ms[li - 1])] = (2 * e * e - 2 * e) * Ed2
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "const_2layer_moments.json")
    with open(path, "w") as f:
        json.dump(res, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
