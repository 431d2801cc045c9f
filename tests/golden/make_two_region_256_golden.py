"""Write the oracle's scalar flux for the benchmark workload to a golden file.

Workload: 2D unit square, 256x256 jittered points (support 2h, linear RK),
level-symmetric S8 (40 directions), sigma_t = 100 in [0.4, 0.6]^2 and 1
elsewhere, sigma_s = 0.9 sigma_t, q = 1 for x < 0.5, vacuum boundaries,
dt = 0.005, 20 backward-Euler steps from Psi = 0 (Sec. 4.1-4.2).

Only the oracle (plain FP64: exact sparse-LU inner solves, the paper's
unpreconditioned outer GMRES to 1e-13) and the seeded input generator are
used; nothing here loads the CUDA library.  The file keeps the point values
phi_i = sum_j V_j U_j(x_i) Phi_j (Eq. flux-expansion) after steps 1, 10 and
20, and the outer iteration count of every step.

Run from the repository root:  python tests/golden/make_two_region_256_golden.py
(about an hour on one core and ~40 GB of host memory: 40 sparse LU factors).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import mlpg_inputs as mi  # noqa: E402
import oracle.mlpg_oracle as O  # noqa: E402

OUT = os.path.join(HERE, "two_region_256_phi.npz")
KEEP = (1, 10, 20)


def main(n_per_dim=256, out=OUT):
    prob = mi.two_region_2d(n_per_dim=n_per_dim)
    t0 = time.time()
    disc = O.Discretization(prob.x, prob.R, prob.lo, prob.hi)
    F = disc.assemble_per_point(prob.sigma_t, prob.sigma_s, prob.q)
    tr = O.Transport(disc, F, prob.omega, prob.w, psi_b=prob.inflow)
    sol = O.Solver(tr, outer_tol=1e-13)
    interp = disc.interpolation_matrix()
    Psi = np.zeros((tr.M, disc.n))
    Phi = tr.D(Psi)
    keep, outer = {}, []
    for k in range(1, prob.steps + 1):
        Psi, Phi, st = sol.step(Psi, prob.dt, Phi_guess=Phi)
        outer.append(st.outer_iterations)
        if k in KEEP:
            keep[f"phi_{k}"] = interp @ Phi
        print(f"step {k}: outer {st.outer_iterations}, residual {st.outer_residual:.2e}, "
              f"{time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(out, n_per_dim=n_per_dim, steps=prob.steps, outer_iterations=np.array(outer),
                        **keep)
    print("wrote", out)


if __name__ == "__main__":
    main()
