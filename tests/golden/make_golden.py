"""Write tests/golden/h_closed_forms.txt from the oracle (exact rationals).

The table holds the rational parts of the paper's closed forms H_1 and H_2
(Appendix A.1, the two displays after eq:Fullint) for |alpha| <= 12:
    H_c(alpha; lambda) = (num/den) / (2 pi) * (2 lambda^2)^{-(n+1)},
    n = (alpha_1 + alpha_2 - 1) / 2.
Only oracle/ is called.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.coefficients import _h_rational  # noqa: E402

out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "h_closed_forms.txt")
with open(out, "w") as f:
    f.write("# Rational parts of H_1 (comp 1) and H_2 (comp 2), |alpha| <= 12.\n")
    f.write("# Source: arXiv:1010.2475, Appendix A.1, closed forms after eq:Fullint.\n")
    f.write("# H_c = num/den / (2 pi) * (2 lambda^2)^(-(n+1)), n = (a1 + a2 - 1)/2.\n")
    f.write("# columns: comp a1 a2 num den\n")
    for comp in (1, 2):
        for n in range(13):
            for a2 in range(n + 1):
                a1 = n - a2
                r = _h_rational(a1, a2, comp)
                f.write(f"{comp} {a1} {a2} {r.numerator} {r.denominator}\n")
print("wrote", out)
