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


# Hopf-Lax closed forms (Section 2: phi(x, t) = min_y J(y) + t H*((x - y)/t),
# with H* the indicator of the dual unit ball) for c = 0, c0 = 0 and small
# hand-checkable x:
#   kind 0: J = 1/2|x|^2,     H = |.|_inf: phi = 1/2 |x - pi(x)|^2, grad = x - pi(x),
#           pi = projection on the l1 ball of radius t;
#   kind 1: J = 1/2|x|_inf^2, H = |.|_1:   phi = 1/2 m^2, m = max_i (|x_i| - t)_+,
#           grad = m sign(x_i*) e_i* (i* the unique maximiser);
#   kind 2: J = 1/2|x|_1^2,   H = |.|_inf: phi = 1/2 (|x|_1 - t)_+^2,
#           grad = (|x|_1 - t)_+ sign(x) (no zero coordinate).
NORM_CASES = [  # (kind, x, t)
    (0, [3.0, 1.0], 1.0),         # pi = (1, 0): phi = 2.5, grad = (2, 1)
    (0, [3.0, -3.0], 2.0),        # pi = (1, -1): phi = 4, grad = (2, -2)
    (0, [0.5, -0.25], 1.0),       # inside the ball: phi = 0, grad = 0
    (0, [4.0, 2.0, -1.0], 3.0),   # pi = (2.5, 0.5, 0): phi = 2.75
    (1, [3.0, -1.0, 0.5], 1.0),   # m = 2: phi = 2, grad = (2, 0, 0)
    (1, [-4.0, 2.5], 0.5),        # m = 3.5: phi = 6.125, grad = (-3.5, 0)
    (2, [2.0, -1.0], 1.0),        # |x|_1 - t = 2: phi = 2, grad = (2, -2)
    (2, [1.0, 2.0, -0.5], 0.5),   # 3: phi = 4.5, grad = (3, 3, -3)
]


def l1ball_projection(x, r):
    """Projection on {|z|_1 <= r} by the sorted-breakpoint rule."""
    if np.abs(x).sum() <= r:
        return x.copy()
    u = np.sort(np.abs(x))[::-1]
    css = np.cumsum(u)
    k = np.nonzero(u * np.arange(1, len(u) + 1) > (css - r))[0][-1]
    mu = (css[k] - r) / (k + 1.0)
    return np.sign(x) * np.maximum(np.abs(x) - mu, 0)


def norm_rows():
    rows = []
    for kind, x, t in NORM_CASES:
        x = np.array(x)
        if kind == 0:
            g = x - l1ball_projection(x, t)
            phi = 0.5 * g @ g
        elif kind == 1:
            e = np.maximum(np.abs(x) - t, 0)
            i = int(np.argmax(e))
            phi = 0.5 * e[i] ** 2
            g = np.zeros_like(x)
            g[i] = e[i] * np.sign(x[i])
        else:
            m = max(np.abs(x).sum() - t, 0.0)
            phi = 0.5 * m * m
            g = m * np.sign(x)
        rows.append((kind, x, t, phi, g))
    return rows


def write_norms():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "section4_norm_kinds.txt")
    with open(out, "w") as f:
        f.write("# Hopf-Lax closed forms for the norm kinds of Sections 4.2-4.4 (c = 0, c0 = 0).\n")
        f.write("# kind 0: J = 1/2|x|^2, H = l_inf; kind 1: J = 1/2|x|_inf^2, H = l1; kind 2: J = 1/2|x|_1^2, H = l_inf\n")
        f.write("# columns: kind n x(n) t phi grad(n); written by tests/golden/make_golden.py\n")
        for kind, x, t, phi, g in norm_rows():
            vals = [kind, len(x)] + list(x) + [t, phi] + list(g)
            f.write(" ".join(repr(float(v)) for v in vals) + "\n")


if __name__ == "__main__":
    main()
    write_norms()
