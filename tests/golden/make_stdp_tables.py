"""Write stdp_q16_tables.txt: the STDP pair rule of the paper (Sec. 2,
"Synaptic update" equation) at integer lags, rounded to Q16.

    LTP(k) = round(A+ * exp(-k / tau+) * 65536),  A+ = 0.1 mV,  tau+ = 20 ms
    LTD(k) = round(A- * exp(-k / tau-) * 65536),  A- = 0.12 mV, tau- = 20 ms

evaluated with 50-digit arithmetic (mpmath) so the rounding is exact; halves
round away from zero.  Independent of both the oracle and the CUDA path.
Run:  python tests/golden/make_stdp_tables.py
"""
import os

import mpmath

mpmath.mp.dps = 50


def q16(amplitude, tau, k):
    x = mpmath.mpf(amplitude) * mpmath.e ** (-mpmath.mpf(k) / mpmath.mpf(tau)) * 65536
    return int(mpmath.floor(x + mpmath.mpf("0.5")))


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "stdp_q16_tables.txt")
    with open(out, "w") as f:
        f.write("# STDP pair rule (paper Sec. 2, 'Synaptic update' equation) in Q16 at lag k ms\n")
        f.write("# A+ = 0.1 mV, A- = 0.12 mV, tau+ = tau- = 20 ms; written by make_stdp_tables.py\n")
        f.write("# k ltp_q16 ltd_q16\n")
        for k in range(256):
            f.write("%d %d %d\n" % (k, q16("0.1", 20, k), q16("0.12", 20, k)))


if __name__ == "__main__":
    main()
