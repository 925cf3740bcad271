"""FP64 oracle of the geometry-updated time stepping (test infrastructure only: only
tests/, the smoke check and the benchmark's CPU arm load it).

Section 2.3 writes the structural system as M u'' + C u' + K(u) u = f, updates the lumen
geometry by the displacement at every step, re-assembles the stiffness only after a
prescribed number of iterations, and keeps the lumped mass fixed. Reading (the paper gives
no formula): K(u) is the stiffness of the current surface, applied to displacement
increments, and the internal force is accumulated along the path. With re-assembly every k
steps on the surface X + u_m (m a multiple of k), the step from u_n uses

    f_int(u_n) = f_int(u_m) + K(X + u_m) (u_n - u_m),        f_int(u_0) = 0 at rest,

each realisation on its own deformed surface, with the same (E h)_e,s; masses and the
traction history stay those of the reference geometry. Without re-assembly this is the
linear method. (Multiplying the total displacement by the re-assembled stiffness instead,
K(X + u_m) u_n, is not objective: on the configuration's tube it left the fixed point and
inverted elements within a few thousand steps even at 2 kPa.)

Each realisation is stepped on its own (realisations are independent), with the linear
oracle's pieces: element matrices (oracle.element_matrices) rebuilt on the deformed
coordinates, the internal force (Model.internal_force) and the central-difference steps
(Model.steps). Writing f_int(u_n) = K_m u_n + c_m with c_m = f_int(u_m) - K_m u_m, the
steps see the stiffness K_m and the load f_n - c_m, which the oracle passes as one extra
traction pattern -c_m with amplitude 1.
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
        modes0, amp0 = mod.modes, mod.amp
        up, uc = mod.start()
        c = None                                   # c_m [1][N][3]; None before the first re-assembly
        step = 0
        while step < n_steps:
            if step > 0 and step % k == 0:
                f_int = mod.internal_force(uc) + (0.0 if c is None else c)   # f_int(u_m), old stiffness
                K, _ = element_matrices(mesh.xyz + uc[0], mesh.tri, case["nu"], case["kshear"])
                mod.Kg = np.ascontiguousarray(K.reshape(mod.E, 81))
                c = f_int - mod.internal_force(uc)                          # new stiffness
                mod.modes = np.ascontiguousarray(np.concatenate([modes0, -c], axis=0))
                mod.amp = np.ascontiguousarray(np.concatenate([amp0, np.ones((amp0.shape[0], 1))], axis=1))
                mod.J = mod.modes.shape[0]
            m = min(k - step % k, n_steps - step)
            mod.steps(up, uc, step, m)
            step += m
        out[j] = uc[0]
    return out
