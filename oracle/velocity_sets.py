"""Velocity sets of the oracle, typed from the paper's tables (FP64).

TEST INFRASTRUCTURE ONLY.  Nothing under ``oracle/`` is part of the product
path: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The CUDA library holds its own, independently
typed copy of these tables.

Sources (section / table of arXiv:2101.03982):

* D2Q9, D3Q27: Gauss-Hermite product rules of D1Q3 (Sec. 2, Table 1).  With the
  weight function of Sec. 2 (unit variance) the 1D nodes are the roots of He_3,
  0 and +-sqrt(3), with weights 2/3, 1/6, 1/6.
* D2Q25: product rule of D1Q5, the roots of He_5: 0, +-sqrt(5 -+ sqrt(10)),
  weights 8/15 and (7 +- 2 sqrt(10))/60 (Sec. 2, Table 1).
* D2Q19: Appendix C (Haegemans-Piessens cubature).
* D3Q13: Table 2 (icosahedron).  D3Q21: Table 3 (dodecahedron, c_s = sqrt(3/5)).
* D3V27: Appendix D (Stroud-Secrest, degree 7).
* D3Q45: Appendix E (Konyaev cubature), the 45 printed rows in printed order.

Ordering convention (shared by the CUDA tables, which are typed separately):
rows in printed order, orbit by orbit; inside a printed row with +- signs the
signs of the nonzero components are enumerated left to right, leftmost slowest,
+ before -; a row marked "(cyc)" is followed by its images with the components
shifted right by one and then by two positions ((a,b,c) -> (c,a,b) -> (b,c,a)).
Product sets use i = ix + q*iy (+ q*q*iz) over the 1D node order
[0, +a1, -a1, +a2, -a2].
"""
import itertools
import math

import numpy as np

PHI = (1.0 + math.sqrt(5.0)) / 2.0


def _signed_orbit(row, images=1):
    """Enumerate a printed row with +- signs (and optional cyclic images)."""
    out = []
    base = list(row)
    for k in range(images):
        img = base[len(base) - k:] + base[:len(base) - k] if k else list(base)
        nz = [a for a in range(len(img)) if img[a] != 0.0]
        for signs in itertools.product((1.0, -1.0), repeat=len(nz)):
            v = list(img)
            for a, s in zip(nz, signs):
                v[a] = s * img[a]
            out.append(v)
    return out


def _product(nodes, weights, dim):
    q = len(nodes)
    xi, w = [], []
    for idx in itertools.product(range(q), repeat=dim):
        # idx is (iz, iy, ix) order of itertools; we want x fastest.
        rev = idx[::-1]
        xi.append([nodes[rev[a]] for a in range(dim)])
        w.append(math.prod(weights[rev[a]] for a in range(dim)))
    return np.array(xi, dtype=np.float64), np.array(w, dtype=np.float64)


def _d1q3():
    a = math.sqrt(3.0)
    return [0.0, a, -a], [2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0]


def _d1q5():
    s10 = math.sqrt(10.0)
    a1, a2 = math.sqrt(5.0 - s10), math.sqrt(5.0 + s10)
    w1, w2 = (7.0 + 2.0 * s10) / 60.0, (7.0 - 2.0 * s10) / 60.0
    return [0.0, a1, -a1, a2, -a2], [8.0 / 15.0, w1, w1, w2, w2]


def _d2q19():
    rows = [
        (0.3168437267921905, [0.0, 0.0]),
        (0.10558878375062891, [1.4869982213169028, 0.0]),
        (0.1024247123210936, [0.775196278121181, 1.367469636752619]),
        (0.00953510698543825, [2.5175897644357486, 1.105629214668943]),
        (0.006865104210104631, [0.0, 2.9213306655318734]),
        (0.002405335328939458, [1.8663975507141328, 2.6987507639352253]),
        (0.0003939393722285871, [3.8358342053914734, 0.0]),
    ]
    xi, w = [], []
    for wt, r in rows:
        for v in _signed_orbit(r):
            xi.append(v)
            w.append(wt)
    return np.array(xi), np.array(w)


def _d3q13():
    r = math.sqrt((5.0 + math.sqrt(5.0)) / 2.0)
    s = math.sqrt((5.0 - math.sqrt(5.0)) / 2.0)
    xi, w = [[0.0, 0.0, 0.0]], [2.0 / 5.0]
    for row in ([0.0, r, s], [s, 0.0, r], [r, s, 0.0]):
        for v in _signed_orbit(row):
            xi.append(v)
            w.append(1.0 / 20.0)
    return np.array(xi), np.array(w)


def _d3q21():
    xi, w = [[0.0, 0.0, 0.0]], [2.0 / 5.0]
    for row in ([1.0, 1.0, 1.0], [0.0, PHI, 1.0 / PHI], [1.0 / PHI, 0.0, PHI],
                [PHI, 1.0 / PHI, 0.0]):
        for v in _signed_orbit(row):
            xi.append(v)
            w.append(3.0 / 100.0)
    return np.array(xi), np.array(w)


def _d3v27():
    a, b, c = 1.1198362860638005, 2.358709038202103, 3.142130383387586
    xi, w = [[0.0, 0.0, 0.0]], [0.31247897198654906]
    for v in _signed_orbit([a, a, a]):
        xi.append(v)
        w.append(0.06338446047675325)
    for v in _signed_orbit([b, 0.0, 0.0], images=3):
        xi.append(v)
        w.append(0.029035130153906134)
    for v in _signed_orbit([c, c, 0.0], images=3):
        xi.append(v)
        w.append(0.0005195469396656799)
    return np.array(xi), np.array(w)


_D3Q45_ROWS = """
0.20740740740740618 0.0 0.0 0.0
0.05787037037037047 0.06386083877343968 -1.2239121278243665 -1.2239121278243665
0.05787037037037047 -0.06386083877343968 1.2239121278243665 1.2239121278243665
0.05787037037037047 1.2239121278243665 -0.06386083877343968 1.2239121278243665
0.05787037037037047 -1.2239121278243665 0.06386083877343968 -1.2239121278243665
0.05787037037037047 1.2239121278243665 1.2239121278243665 -0.06386083877343968
0.05787037037037047 -1.2239121278243665 -1.2239121278243665 0.06386083877343968
0.05787037037037047 1.5766994272507744 -0.5069610024977665 -0.5069610024977665
0.05787037037037047 -1.5766994272507744 0.5069610024977665 0.5069610024977665
0.05787037037037047 0.5069610024977665 0.5069610024977665 -1.5766994272507744
0.05787037037037047 -0.5069610024977665 -0.5069610024977665 1.5766994272507744
0.05787037037037047 -0.5069610024977665 1.5766994272507744 -0.5069610024977665
0.05787037037037047 0.5069610024977665 -1.5766994272507744 0.5069610024977665
0.00462962962962958 2.403092127540177 0.8892242114059369 -1.5602655313772367
0.00462962962962958 -2.403092127540177 -0.8892242114059369 1.5602655313772367
0.00462962962962958 -2.403092127540177 1.5602655313772367 -0.8892242114059369
0.00462962962962958 2.403092127540177 -1.5602655313772367 0.8892242114059369
0.00462962962962958 -0.8892242114059369 -2.403092127540177 1.5602655313772367
0.00462962962962958 0.8892242114059369 2.403092127540177 -1.5602655313772367
0.00462962962962958 -0.8892242114059369 1.5602655313772367 -2.403092127540177
0.00462962962962958 0.8892242114059369 -1.5602655313772367 2.403092127540177
0.00462962962962958 -1.5602655313772367 0.8892242114059369 2.403092127540177
0.00462962962962958 -1.5602655313772367 2.403092127540177 0.8892242114059369
0.00462962962962958 1.5602655313772367 -0.8892242114059369 -2.403092127540177
0.00462962962962958 1.5602655313772367 -2.403092127540177 -0.8892242114059369
0.00462962962962958 0.4744978678080795 0.4744978678080795 2.9239876105912574
0.00462962962962958 0.4744978678080795 2.9239876105912574 0.4744978678080795
0.00462962962962958 -0.4744978678080795 -0.4744978678080795 -2.9239876105912574
0.00462962962962958 -0.4744978678080795 -2.9239876105912574 -0.4744978678080795
0.00462962962962958 2.9239876105912574 0.4744978678080795 0.4744978678080795
0.00462962962962958 -2.9239876105912574 -0.4744978678080795 -0.4744978678080795
0.00462962962962958 1.7320508075688787 1.7320508075688787 1.7320508075688787
0.00462962962962958 -1.7320508075688787 -1.7320508075688787 -1.7320508075688787
0.0004629629629629939 -2.7367507163016924 0.14279717659756475 -2.7367507163016924
0.0004629629629629939 2.7367507163016924 2.7367507163016924 -0.14279717659756475
0.0004629629629629939 2.7367507163016924 -0.14279717659756475 2.7367507163016924
0.0004629629629629939 -2.7367507163016924 -2.7367507163016924 0.14279717659756475
0.0004629629629629939 0.14279717659756475 -2.7367507163016924 -2.7367507163016924
0.0004629629629629939 -0.14279717659756475 2.7367507163016924 2.7367507163016924
0.0004629629629629939 -3.5256070994177073 1.1335992635264445 1.1335992635264445
0.0004629629629629939 3.5256070994177073 -1.1335992635264445 -1.1335992635264445
0.0004629629629629939 1.1335992635264445 -3.5256070994177073 1.1335992635264445
0.0004629629629629939 -1.1335992635264445 3.5256070994177073 -1.1335992635264445
0.0004629629629629939 1.1335992635264445 1.1335992635264445 -3.5256070994177073
0.0004629629629629939 -1.1335992635264445 -1.1335992635264445 3.5256070994177073
"""


def _d3q45():
    data = np.array([[float(t) for t in ln.split()] for ln in _D3Q45_ROWS.strip().splitlines()])
    return data[:, 1:].copy(), data[:, 0].copy()


class VelocitySet:
    """Abscissae xi (Q, D), weights w (Q,), speed of sound cs, claimed degree d."""

    def __init__(self, name, xi, w, cs, degree):
        self.name = name
        self.xi = np.asarray(xi, dtype=np.float64)
        self.w = np.asarray(w, dtype=np.float64)
        self.cs = float(cs)
        self.degree = int(degree)

    @property
    def Q(self):
        return self.xi.shape[0]

    @property
    def D(self):
        return self.xi.shape[1]

    def scaled(self, s):
        """Rescale abscissae and speed of sound by s (same weights)."""
        return VelocitySet(self.name, self.xi * s, self.w, self.cs * s, self.degree)


def get(name):
    """Velocity set by name, with c_s as the paper tabulates it."""
    name = name.upper()
    if name == "D2Q9":
        xi, w = _product(*_d1q3(), 2)
        return VelocitySet(name, xi, w, 1.0, 5)
    if name == "D3Q27":
        xi, w = _product(*_d1q3(), 3)
        return VelocitySet(name, xi, w, 1.0, 5)
    if name == "D2Q25":
        xi, w = _product(*_d1q5(), 2)
        return VelocitySet(name, xi, w, 1.0, 9)
    if name == "D2Q19":
        return VelocitySet(name, *_d2q19(), 1.0, 9)
    if name == "D3Q13":
        return VelocitySet(name, *_d3q13(), 1.0, 5)
    if name == "D3Q21":
        return VelocitySet(name, *_d3q21(), math.sqrt(3.0 / 5.0), 5)
    if name == "D3V27":
        return VelocitySet(name, *_d3v27(), 1.0, 7)
    if name == "D3Q45":
        return VelocitySet(name, *_d3q45(), 1.0, 9)
    raise KeyError(name)


ALL_SETS = ("D2Q9", "D2Q19", "D2Q25", "D3Q13", "D3Q21", "D3Q27", "D3V27", "D3Q45")
