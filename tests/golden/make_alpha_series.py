"""Writes alpha_series.txt: the alpha/beta series of Sec. 2 in 50-digit decimal arithmetic.

alpha_0 = 1, alpha_{k+1} = (1 + sqrt(4 alpha_k^2 + 1)) / 2 and
beta_k = (alpha_k - 1) / alpha_{k+1} are evaluated with Python's `decimal`
module, independently of the oracle's float64 code, and rounded to 10 places.
The first values also have closed forms (alpha_1 is the golden ratio).
"""
import os
from decimal import Decimal, getcontext

getcontext().prec = 50
a = [Decimal(1)]
for _ in range(6):
    a.append((1 + (4 * a[-1] * a[-1] + 1).sqrt()) / 2)
lines = ["# alpha_k of Sec. 2 (alpha_0 = 1, alpha_{k+1} = (1 + sqrt(4 alpha_k^2 + 1)) / 2)",
         "# and beta_k = (alpha_k - 1) / alpha_{k+1}; written by make_alpha_series.py in",
         "# 50-digit decimal arithmetic. Closed forms: alpha_1 = (1 + sqrt 5) / 2,",
         "# alpha_2 = (1 + sqrt(7 + 2 sqrt 5)) / 2, beta_1 = (sqrt 5 - 1) / (1 + sqrt(7 + 2 sqrt 5)).",
         "# k  alpha_k        beta_k"]
for k in range(5):
    lines.append(f"{k}  {a[k]:.10f}   {(a[k] - 1) / a[k + 1]:.10f}")
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "alpha_series.txt"), "w") as f:
    f.write("\n".join(lines) + "\n")
