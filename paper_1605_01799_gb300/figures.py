"""The paper's 2-D slices (Section 4.5, Figs. 1-5) computed with the GPU solver.

phi((x1, x2, 0, ..., 0), t) in dimension n = 8 on a 100 x 100 grid of
[-20, 20]^2 (x_i = -20 + 40 k / 99, k = 0..99), at four times, for

    fig1  J = 1/2|x|_inf^2,   H = |p|_2                      t = 0, 5, 10, 15
    fig2  J = 1/2|x|_1^2,     H = |p|_1                      t = 0, 5, 10, 15
    fig3  J = 1/2|x|_1^2,     H = sqrt(<p, D p>)              t = 0, 5, 10, 15
    fig4  J = min(1/2|x|^2 - <b, x>, 1/2|x|^2 + <b, x>),
          b = (1, ..., 1), H = |p|_1  (minimum over initial data)  t = 0, 5, 10, 15
    fig5  J = 1/2|x|_1^2,     H = min(|p|_1, sqrt(<p, 4/3 D p>))
          (maximum over Hamiltonians)                          t = 2, 5, 9, 12

with D_ii = 1 + (i-1)/(n-1).  The figures themselves are images in the paper;
here each slice is a plain array: ``slices()`` returns them and ``write()``
stores each as .npy plus an 8-bit greyscale PGM (a plain-text header and
raw bytes, no graphics library), with the paper's level-line spacing marked
in black.

    python -m paper_1605_01799_gb300.figures --out DIR
"""
import argparse
import os

import numpy as np

N = 8
GRID = 100
TIMES = {"fig1": (0.0, 5.0, 10.0, 15.0), "fig2": (0.0, 5.0, 10.0, 15.0), "fig3": (0.0, 5.0, 10.0, 15.0),
         "fig4": (0.0, 5.0, 10.0, 15.0), "fig5": (2.0, 5.0, 9.0, 12.0)}
LEVEL_STEP = {"fig1": 5.0, "fig2": 20.0, "fig3": 20.0, "fig4": 15.0, "fig5": 15.0}


def grid_points(grid=GRID, n=N):
    """The query points (x1, x2, 0, ..., 0), x2 fastest: [grid * grid, n]."""
    g = -20.0 + 40.0 * np.arange(grid) / (grid - 1)
    X = np.zeros((grid * grid, n))
    X[:, 0] = np.repeat(g, grid)
    X[:, 1] = np.tile(g, grid)
    return X


def _D(n=N):
    return 1.0 + np.arange(n) / (n - 1.0)


def _common(hg):
    return dict(tol=1e-12, max_iter=100000, precision=hg.P_FP32, stop_rule=hg.STOP_UREL, c0=0.0)


def _solver(fig, hg):
    """A function (x [B, n] float32 cuda, t [B] float32 cuda) -> phi [B]."""
    kw = _common(hg)
    if fig == "fig1":
        h = hg.Hopf(None, hg.H_L2, j_kind=hg.J_LINFSQ, n=N, **kw)
        return lambda x, t: h.eval(x, t)["phi"], [h]
    if fig == "fig2":
        h = hg.Hopf(None, hg.H_L1, j_kind=hg.J_L1SQ, n=N, **kw)
        return lambda x, t: h.eval(x, t)["phi"], [h]
    if fig == "fig3":
        h = hg.Hopf(None, hg.H_DNORM, w=_D(), j_kind=hg.J_L1SQ, n=N, **kw)
        return lambda x, t: h.eval(x, t)["phi"], [h]
    if fig == "fig4":
        # 1/2|x|^2 -+ <b, x> = 1/2|x -+ b|^2 - 1/2|b|^2: centre +-b, c0 = |b|^2 / 2
        b = np.ones(N)
        kw4 = dict(kw, c0=0.5 * b @ b)
        parts = [hg.Hopf(np.ones(N), hg.H_L1, centre=s * b, **kw4) for s in (1.0, -1.0)]
        return lambda x, t: hg.union_eval(parts, x, t)["phi"], parts
    if fig == "fig5":
        parts = [hg.Hopf(None, hg.H_L1, j_kind=hg.J_L1SQ, n=N, **kw),
                 hg.Hopf(None, hg.H_DNORM, w=4.0 / 3.0 * _D(), j_kind=hg.J_L1SQ, n=N, **kw)]
        return lambda x, t: hg.maxH_eval(parts, x, t)["phi"], parts
    raise ValueError(fig)


def slices(figs=tuple(TIMES), grid=GRID):
    """{fig: [len(times), grid, grid] float64} of phi on the slice (rows x1,
    columns x2)."""
    import torch
    import paper_1605_01799_gb300 as hg
    X = grid_points(grid)
    x = torch.tensor(X, dtype=torch.float32, device="cuda")
    out = {}
    for fig in figs:
        fn, keep = _solver(fig, hg)
        planes = []
        for t in TIMES[fig]:
            tt = torch.full((X.shape[0],), t, dtype=torch.float32, device="cuda")
            planes.append(fn(x, tt).cpu().numpy().reshape(grid, grid))
        out[fig] = np.stack(planes)
        for h in keep:
            h.close()
    return out


def to_pgm(phi, step):
    """8-bit greyscale of phi (min black .. max white) with the multiples of
    ``step`` drawn as black level lines (cells whose 2 x 2 neighbourhood
    crosses one)."""
    lo, hi = float(phi.min()), float(phi.max())
    img = np.zeros(phi.shape, np.uint8) if hi <= lo else np.round(255 * (phi - lo) / (hi - lo)).astype(np.uint8)
    k = np.floor(phi / step)
    line = np.zeros(phi.shape, bool)
    line[:-1, :] |= k[:-1, :] != k[1:, :]
    line[:, :-1] |= k[:, :-1] != k[:, 1:]
    img[line] = 0
    return img


def write(out_dir, figs=tuple(TIMES), grid=GRID):
    os.makedirs(out_dir, exist_ok=True)
    res = slices(figs, grid)
    paths = []
    for fig, planes in res.items():
        np.save(os.path.join(out_dir, fig + ".npy"), planes)
        for t, phi in zip(TIMES[fig], planes):
            p = os.path.join(out_dir, "%s_t%g.pgm" % (fig, t))
            img = to_pgm(phi, LEVEL_STEP[fig])
            with open(p, "wb") as f:
                f.write(b"P5\n%d %d\n255\n" % (img.shape[1], img.shape[0]))
                f.write(img[::-1].tobytes())  # x1 upwards
            paths.append(p)
    return paths


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", default="figures_out")
    ap.add_argument("--grid", type=int, default=GRID)
    a = ap.parse_args()
    for p in write(a.out, grid=a.grid):
        print(p)


if __name__ == "__main__":
    main()
