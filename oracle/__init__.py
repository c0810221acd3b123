"""Plain fp64 CPU oracle for range-separated stochastic-RI GF2 (RS-SRI-GF2).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
package: only the tests, the smoke check and the CPU-baseline leg of the
benchmark use it.  It shares no code with the CUDA library; the two meet only
through seeded input arrays and each side's own implementation of the
published SplitMix64 generator.

Every function follows one equation of the paper (Dou, Chen, Takeshita, Baer,
Neuhauser, Rabani, "Range-Separated Stochastic Resolution of Identity",
arXiv:2005.12338) and is written for a reader to check against it by eye,
not for speed.  Where the paper is ambiguous the reading taken is named in the
docstring.

Pins (tests marked "not gpu") tie the oracle to things other than itself:
SplitMix64's published output stream, the brute-force O(N^5) definition of
Eq. 20 on full 4-index integrals, the closed-form MP2 energy reached by the
tau quadrature of Eq. 26, exhaustive enumeration of all Rademacher vectors,
the RI limit at eps = eps' = 0 (Sec. II), the SRI limit with an empty large
part, the 1/sqrt(N_s) error law (Sec. IV), the G(tau) jump and particle-number
relations (Eq. 2 and Sec. III), and hand-worked screening/cut fixtures.
"""
from .rssri import *  # noqa: F401,F403
from .rng import splitmix64_stream, splitmix64_first, rademacher  # noqa: F401
