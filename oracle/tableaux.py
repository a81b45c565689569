"""Butcher tableaux of the IMEX Runge-Kutta methods, as exact rationals.

TEST INFRASTRUCTURE ONLY: the oracle is imported by the tests, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``.
Nothing on the product path may import it.

Source: the appendix of the paper ("Butcher tableaux of the IMEX Runge-Kutta
methods"), one subsection per method, and the CK structure of Eq.
(imex-rk:butcher) in Sec. 2.2: shared nodes ``c``, ``a^IM_11 = 0``, a DIRK
implicit part and an ERK explicit part with ``s`` stages each.  Table 1 lists
the stage counts, orders and the SA / FSAL properties checked by the tests.

``IMEX-EULER`` is the first-order IMEX Euler rule that Sec. 2.2 uses to start
BDF2 and Sec. 2.4 / Sec. 3.2.3 use as the SDC predictor, written as a two-stage
CK tableau (explicit Euler for f_c, implicit Euler for f_d).
"""
from fractions import Fraction as Fr


class Tableau:
    """c, A^IM, b^IM, A^EX, b^EX of one CK-type IMEX RK method (Eq. imex-rk:butcher)."""

    def __init__(self, name, c, AI, bI, AE, bE, order):
        self.name = name
        self.s = len(c)
        self.c = [Fr(x) for x in c]
        self.AI = [[Fr(x) for x in row] for row in AI]
        self.bI = [Fr(x) for x in bI]
        self.AE = [[Fr(x) for x in row] for row in AE]
        self.bE = [Fr(x) for x in bE]
        self.order = order

    def as_float(self):
        """The coefficients of Eq. (imex-rk:butcher) as floats: c, A^IM, b^IM, A^EX, b^EX."""
        f = float
        return ([f(x) for x in self.c], [[f(x) for x in r] for r in self.AI],
                [f(x) for x in self.bI], [[f(x) for x in r] for r in self.AE],
                [f(x) for x in self.bE])


def _lower(rows, s):
    """Pad lower-triangular row lists to a full s x s matrix."""
    out = []
    for r in rows:
        out.append(list(r) + [0] * (s - len(r)))
    return out


def _F(p, q):
    """The exact rational p / q of a printed coefficient."""
    return Fr(p, q)


# RK-TR: 3-stage IMEX trapezoidal rule (appendix, RK-TR).
RK_TR = Tableau(
    "TR",
    c=[0, 1, 1],
    AI=_lower([[0], [0, 1], [_F(1, 2), 0, _F(1, 2)]], 3),
    bI=[_F(1, 2), 0, _F(1, 2)],
    AE=_lower([[0], [1, 0], [_F(1, 2), _F(1, 2), 0]], 3),
    bE=[_F(1, 2), _F(1, 2), 0],
    order=2)

# RK-CB2 (appendix, RK-CB2).
RK_CB2 = Tableau(
    "CB2",
    c=[0, _F(2, 5), 1],
    AI=_lower([[0], [0, _F(2, 5)], [0, _F(5, 6), _F(1, 6)]], 3),
    bI=[0, _F(5, 6), _F(1, 6)],
    AE=_lower([[0], [_F(2, 5), 0], [0, 1, 0]], 3),
    bE=[0, _F(5, 6), _F(1, 6)],
    order=2)

# RK-CB3c (appendix, RK-CB3c), used as printed there.
_c2 = _F(3375509829940, 4525919076317)
_c3 = _F(272778623835, 1039454778728)
_b2 = _F(673488652607, 2334033219546)
_b3 = _F(493801219040, 853653026979)
_b4 = _F(184814777513, 1389668723319)
RK_CB3C = Tableau(
    "CB3c",
    c=[0, _c2, _c3, 1],
    AI=_lower([[0], [0, _c2],
               [0, _F(-11712383888607531889907, 32694570495602105556248),
                _F(566138307881, 912153721139)],
               [0, _b2, _b3, _b4]], 4),
    bI=[0, _b2, _b3, _b4],
    AE=_lower([[0], [_c2, 0], [0, _c3, 0],
               [0, _b2, _F(1660544566939, 2334033219546), 0]], 4),
    bE=[0, _b2, _b3, _b4],
    order=3)

# RK-CB3e (appendix, RK-CB3e).
RK_CB3E = Tableau(
    "CB3e",
    c=[0, _F(1, 3), 1, 1],
    AI=_lower([[0], [0, _F(1, 3)], [0, _F(1, 2), _F(1, 2)],
               [0, _F(3, 4), _F(-1, 4), _F(1, 2)]], 4),
    bI=[0, _F(3, 4), _F(-1, 4), _F(1, 2)],
    AE=_lower([[0], [_F(1, 3), 0], [0, 1, 0], [0, _F(3, 4), _F(1, 4), 0]], 4),
    bE=[0, _F(3, 4), _F(-1, 4), _F(1, 2)],
    order=3)

# RK-CB4 (appendix, RK-CB4).
_a1 = _F(232049084587, 1377130630063)
_a2 = _F(322009889509, 2243393849156)
_a3 = _F(-195109672787, 1233165545817)
_bb4 = _F(-340582416761, 705418832319)
_bb5 = _F(463396075661, 409972144477)
_bb6 = _F(323177943294, 1626646580633)
RK_CB4 = Tableau(
    "CB4",
    c=[0, _F(1, 4), _F(3, 4), _F(3, 8), _F(1, 2), 1],
    AI=_lower([[0],
               [_F(1, 8), _F(1, 8)],
               [_F(216145252607, 961230882893), _F(257479850128, 1143310606989),
                _F(30481561667, 101628412017)],
               [_a1, _F(-381180097479, 1276440792700), _F(-54660926949, 461115766612),
                _F(344309628413, 552073727558)],
               [_a1, _a2, _F(-100836174740, 861952129159), _F(-250423827953, 1283875864443),
                _F(1, 2)],
               [_a1, _a2, _a3, _bb4, _bb5, _bb6]], 6),
    bI=[_a1, _a2, _a3, _bb4, _bb5, _bb6],
    AE=_lower([[0],
               [_F(1, 4), 0],
               [_F(153985248130, 1004999853329), _F(902825336800, 1512825644809), 0],
               [_a1, _F(99316866929, 820744730663), _F(82888780751, 969573940619), 0],
               [_a1, _a2, _F(57501241309, 765040883867), _F(76345938311, 676824576433), 0],
               [_a1, _a2, _a3, _F(-4099309936455, 6310162971841),
                _F(1395992540491, 933264948679), 0]], 6),
    bE=[_a1, _a2, _a3, _bb4, _bb5, _bb6],
    order=4)

# RK-ARS3, the (4,4,3) method of Ascher, Ruuth and Spiteri (appendix, RK-ARS3).
RK_ARS3 = Tableau(
    "ARS3",
    c=[0, _F(1, 2), _F(2, 3), _F(1, 2), 1],
    AI=_lower([[0], [0, _F(1, 2)], [0, _F(1, 6), _F(1, 2)],
               [0, _F(-1, 2), _F(1, 2), _F(1, 2)],
               [0, _F(3, 2), _F(-3, 2), _F(1, 2), _F(1, 2)]], 5),
    bI=[0, _F(3, 2), _F(-3, 2), _F(1, 2), _F(1, 2)],
    AE=_lower([[0], [_F(1, 2), 0], [_F(11, 18), _F(1, 18), 0],
               [_F(5, 6), _F(-5, 6), _F(1, 2), 0],
               [_F(1, 4), _F(7, 4), _F(3, 4), _F(-7, 4), 0]], 5),
    bE=[_F(1, 4), _F(7, 4), _F(3, 4), _F(-7, 4), 0],
    order=3)

# IMEX Euler (Sec. 2.2, starting step of BDF2; Sec. 2.4 SDC predictor).
IMEX_EULER = Tableau(
    "EULER",
    c=[0, 1],
    AI=[[0, 0], [0, 1]],
    bI=[0, 1],
    AE=[[0, 0], [1, 0]],
    bE=[1, 0],
    order=1)

TABLEAUX = {t.name: t for t in (RK_TR, RK_CB2, RK_CB3C, RK_CB3E, RK_CB4, RK_ARS3, IMEX_EULER)}


def get(name):
    """The tableau of the appendix (or IMEX Euler) by name, with or without the "RK-" prefix."""
    key = name.upper().replace("RK-", "")
    for k, t in TABLEAUX.items():
        if k.upper() == key:
            return t
    raise KeyError(name)
