"""Writes section1_l1_ellipsoid.txt: hand-checkable instances of the worked
example of Section 1 (J = 1/2 (sum x_i^2/a_i^2 - 1), H = l1), evaluated with
that example's closed form  phi = -1/2 + sum_{|x_i|>t} 1/2 ((|x_i|-t)/a_i)^2,
d phi/d x_i = shrink_1(x,t)_i / a_i^2.  Uses numpy only (no oracle, no GPU).
Row layout: a_1..a_n, x_1..x_n, t, phi, grad_1..grad_n."""
import os
import numpy as np

CASES = [  # (a, x, t): small values whose results can be checked by hand
    ([1.0, 2.0, 0.5], [3.0, -1.0, 0.2], 1.0),    # shrink = (2, 0, 0): phi = 1.5, grad = (2, 0, 0)
    ([1.0, 2.0, 0.5], [-3.0, 4.0, 1.5], 0.5),    # shrink = (-2.5, 3.5, 1.0)
    ([2.0, 1.0, 1.0], [0.25, -0.25, 0.0], 0.5),  # all inside: phi = -1/2, grad = 0
    ([0.5, 0.5, 4.0], [1.0, -2.0, 8.0], 1.0),    # shrink = (0, -1, 7)
]


def main():
    rows = []
    for a, x, t in CASES:
        a, x = np.array(a), np.array(x)
        s = np.sign(x) * np.maximum(np.abs(x) - t, 0)
        m = np.abs(x) > t
        phi = -0.5 + 0.5 * (((np.abs(x[m]) - t) / a[m]) ** 2).sum()
        rows.append(np.concatenate([a, x, [t, phi], s / a ** 2]))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "section1_l1_ellipsoid.txt")
    with open(out, "w") as f:
        f.write("# Section 1 worked example (H = l1, J = 1/2 (sum x_i^2/a_i^2 - 1)); closed form of that example.\n")
        f.write("# columns: a(3) x(3) t phi grad(3); written by tests/golden/make_golden.py\n")
        for r in rows:
            f.write(" ".join(repr(float(v)) for v in r) + "\n")


if __name__ == "__main__":
    main()
