"""FP64 oracle of the geometry-updated time stepping (test infrastructure only: only
tests/, the smoke check and the benchmark's CPU arm load it).

Section 2.3 writes the structural system as M u'' + C u' + K(u) u = f: the lumen geometry
is updated by the displacement, the stiffness therefore depends on it, and the solver
can re-assemble K only after a prescribed number of iterations, keeping the lumped mass
fixed. Reading (the paper gives no formula): with re-assembly every k steps, the step
from u_n uses K(X + u_m) u_n, where m is the last multiple of k not above n (m = 0 uses
the reference geometry X) and u_n is the total displacement from X; the element
matrices of realisation s are those of its own deformed surface X + u_s,m, scaled by
the same (E h)_e,s; masses and the traction history stay those of the reference
geometry. A k beyond the run is the linear method.

Each realisation is stepped on its own (realisations are independent), with the linear
oracle's element matrices (oracle.element_matrices) rebuilt on the deformed coordinates
and its central-difference steps (oracle.Model.steps) between re-assemblies.
"""
from __future__ import annotations

import numpy as np

from . import Model, element_matrices


def run_updated(case, n_steps: int, k: int, samples=None):
    """u_n [S][N][3] after n_steps from rest, re-assembling every k steps."""
    mesh = case["mesh"]
    picks = list(range(case["E"].shape[1])) if samples is None else list(samples)
    out = np.zeros((len(picks), mesh.n_nodes, 3))
    for j, s in enumerate(picks):
        mod = Model(case, samples=[s])
        up, uc = mod.start()
        step = 0
        while step < n_steps:
            if step > 0 and step % k == 0:
                K, _ = element_matrices(mesh.xyz + uc[0], mesh.tri, case["nu"], case["kshear"])
                mod.Kg = np.ascontiguousarray(K.reshape(mod.E, 81))
            m = min(k - step % k, n_steps - step)
            mod.steps(up, uc, step, m)
            step += m
        out[j] = uc[0]
    return out
