"""Logical-error-rate statistics: binomial estimates with Wilson score 95%
intervals (the error bars the decoder's failure counts are reported with)."""
import math


def wilson_interval(failures, shots, z=1.959963984540054):
    """Wilson score interval for a binomial proportion (default 95%)."""
    if shots <= 0:
        return (0.0, 1.0)
    p = failures / shots
    denom = 1.0 + z * z / shots
    centre = (p + z * z / (2 * shots)) / denom
    half = z * math.sqrt(p * (1 - p) / shots + z * z / (4 * shots * shots)) / denom
    return (max(0.0, centre - half), min(1.0, centre + half))


def ler_record(p, failures, shots):
    lo, hi = wilson_interval(failures, shots)
    sigma = math.sqrt(max(failures / shots * (1 - failures / shots), 0.0) / shots) if shots else 0.0
    return {"p": p, "failures": int(failures), "shots": int(shots), "ler": failures / shots if shots else None,
            "ci95": [lo, hi], "sigma": sigma}
