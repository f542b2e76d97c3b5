"""The FP64 work per node and direction of the mixed path, the FP64 part of its roofline
(bench.MIXED_FP64_FLOPS), from each scheme's coefficients in the oracle's tables.

With f+- = (E^ +- A^ Q)/2 the double part of h is (1/2) sum_d (n_{-d} + n_{1+d})
(E^_{p-d} + E^_{p+1+d}) plus the midpoint terms, over the node pairs d whose coefficient
is not zero.  Counted with a fused multiply-add as two:
* node products E^ = mx E + my F: 4 variables x 3;
* midpoint metrics, two of them, from the symmetric Lagrange value of 2, 4, 6 or 8 points
  grouped into pair sums: 4 points 5 (2 sums, the weight 9, a difference, the scale),
  6 points 9, 8 points 12;
* midpoint products mm_x E + mm_y F: 4 x 3 per midpoint value (one mean for one-midpoint
  schemes, both sides for two-midpoint schemes);
* per variable, the midpoint term (one product; two-midpoint: three sums and two products)
  and a sum, a product and a sum per node pair;
* the double and float parts joined and the difference of h: 4 + 4.
"""
import bench
import oracle as O

INTERP = {4: 5, 6: 9, 8: 12}


def test_mixed_fp64_flops_follow_the_scheme_tables():
    for scheme in range(5):
        t = O.scheme_table(scheme)
        nmp = 2 if t["hmid"][1] != 0 else 1
        hn = dict(zip(range(-3, 4), t["hnode"]))
        pairs = sum(1 for d in range(4) if hn.get(-d, 0.0) + hn.get(1 + d, 0.0) != 0.0)   # central part only
        points = 2 * t["r"]
        mid_term = 1 if nmp == 1 else 5
        want = 12 + 2 * INTERP[points] + 12 * nmp + 4 * (mid_term + 3 * pairs) + 8
        assert bench.MIXED_FP64_FLOPS[scheme] == want, (scheme, want)
