"""Writes tests/golden/fig2_setups.txt from the oracle only (O1 quadrature).

Setups of Sec. 3.2.1 / Fig. 2: flat Om0 = 0.3, OL0 = 0.7 without radiation
and with Or0 = 1e-5 (then slightly non-flat under closure), H0 = 70 km/s/Mpc,
z1 = 0 and z2 on a logarithmic grid from 1e-3 to 1e3.  The figure's own curves
are not recoverable from the text, so these are oracle values, not the
paper's numbers.
Columns: Or0, z, d_C [Mpc], t [Gyr], X [Mpc], d_M [Mpc], d_L [Mpc], mu [mag].
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import oracle  # noqa: E402

z = np.logspace(-3, 3, 25)
rows = []
for Or in (0.0, 1e-5):
    o = oracle.quad_distances(np.array([70.0, 0.3, 0.7, Or]), z, rtol=1e-15)
    for zi, oi in zip(z, o):
        rows.append([Or, zi, *oi])
out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fig2_setups.txt")
np.savetxt(out, np.array(rows), fmt="%.17g", header=__doc__.strip().replace("\n", " | "))
print(out)
