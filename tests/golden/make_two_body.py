"""Write tests/golden/two_body.txt from the closed form of the two-body
near-field acceleration (Maksimova et al. 2021, Sec. 3.1 near field; Sec. 5.2
Plummer softening): a_1 = G m_2 D / (|D|^2 + eps^2)^(3/2) and
a_2 = -G m_1 D / (|D|^2 + eps^2)^(3/2), D = x_2 - x_1 through the periodic
image chosen by the cell offset. The separations are picked so that
(|D|^2 + eps^2)^(3/2) is an exact rational; the values are computed in exact
rational arithmetic. This script calls neither the oracle nor the CUDA path.

    python tests/golden/make_two_body.py > tests/golden/two_body.txt
"""
from fractions import Fraction as F

HEADER = """# Two-body near-field accelerations derived by hand from the Plummer law
#   a_1 = G m_2 D / (|D|^2 + eps^2)^(3/2),  a_2 = -G m_1 D / (|D|^2 + eps^2)^(3/2),
#   D = x_2 - x_1 taken through the periodic image chosen by the cell offset
# (near field of Maksimova et al. 2021, Sec. 3.1; Plummer softening potential
# of Sec. 5.2). The paper prints no worked example for this path; these rows
# use separations where the closed form is exact in decimal:
#   D = (0.3, 0.4, 0) or (-0.3, 0.4, 0), |D|^2 = 0.25.
#   eps^2 = 0.39 -> s = 0.64, s^(3/2) = 0.512, D/0.512 = (+-0.5859375, 0.78125, 0)
#   eps^2 = 0.75 -> s = 1,    s^(3/2) = 1,     D/1     = (+-0.3, 0.4, 0)
# Columns: L CPD R eps m1 m2  x1 y1 z1  x2 y2 z2  a1x a1y a1z  a2x a2y a2z
# (eps written as sqrt(0.39) = 0.6244997998398398 and sqrt(0.75) = 0.8660254037844386;
#  eps > 0 always: with eps = 0 the self pair would be 0/0)
# Written by tests/golden/make_two_body.py."""

# (comment, L, CPD, R, eps text, eps^2, s^(3/2), m1, m2, x1, x2, D)
ROWS = [
    ("same cell, softened", 5, 5, 2, "0.6244997998398398", F(39, 100), F(512, 1000),
     F(1), F(2), ("1.0", "1.0", "2.5"), ("1.3", "1.4", "2.5"), (F(3, 10), F(4, 10), F(0))),
    ("across the x face (x2 = 4.8 is the image at -0.2), softened", 5, 5, 2, "0.6244997998398398",
     F(39, 100), F(512, 1000), F(3), F(1, 2), ("0.1", "2.5", "2.5"), ("4.8", "2.9", "2.5"),
     (F(-3, 10), F(4, 10), F(0))),
    ("same pair, eps^2 = 0.75: a1 = m2 D, a2 = -m1 D", 5, 5, 2, "0.8660254037844386", F(75, 100),
     F(1), F(3), F(1, 2), ("0.1", "2.5", "2.5"), ("4.8", "2.9", "2.5"), (F(-3, 10), F(4, 10), F(0))),
]


def num(x: F) -> str:
    v = float(x)
    return repr(v) if v != int(v) or abs(v) >= 1e16 else f"{v:.1f}"


def main():
    print(HEADER)
    for comment, L, cpd, R, eps, eps2, s32, m1, m2, x1, x2, D in ROWS:
        assert (sum(d * d for d in D) + eps2) ** 3 == s32 ** 2     # s^(3/2) is exact
        a1 = [m2 * d / s32 for d in D]
        a2 = [-m1 * d / s32 for d in D]
        print(f"# {comment}")
        print(f"{L} {cpd} {R} {eps} {num(m1)} {num(m2)}  {' '.join(x1)}  {' '.join(x2)}  "
              f"{' '.join(num(a) for a in a1)}  {' '.join(num(a) for a in a2)}")


if __name__ == "__main__":
    main()
