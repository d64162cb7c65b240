"""Free-space constants (exact SI definitions used by both sides of every test)."""

import math

MU0 = 4.0e-7 * math.pi
C0 = 299792458.0
EPS0 = 1.0 / (MU0 * C0 * C0)
ETA0 = MU0 * C0
