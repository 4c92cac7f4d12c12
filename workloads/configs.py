"""The named workloads (plain dictionaries, oracle/Config field names).

c1 3x3 chi 8 first order FP64, c2 4x4 off-centre h=2 second order FP32,
c3 64 batched instances, c4 8x8 chi 64 precision study, c5 10x10 chi 100.
"""
import numpy as np

C1 = dict(Lx=3, Ly=3, J=1.0, h=1.0, dt=0.05, order=1, obs=(1, 1), chi_max=8, bp_alpha=0.5,
          bp_tol=1e-10, nsteps=20, precision="fp64")
C2 = dict(Lx=4, Ly=4, J=1.0, h=2.0, dt=0.05, order=2, obs=(1, 1), chi_max=20, bp_alpha=0.5,
          bp_tol=1e-5, nsteps=40, precision="fp32")
C4 = dict(Lx=8, Ly=8, J=1.0, h=2.0, dt=0.05, order=2, obs=(3, 3), chi_max=64, bp_alpha=0.5,
          bp_tol=1e-5, nsteps=60, precision="fp32")
C5 = dict(Lx=10, Ly=10, J=1.0, h=2.0, dt=0.05, order=2, obs=(3, 4), chi_max=100, bp_alpha=0.5,
          bp_tol=1e-5, nsteps=40, precision="fp32")


def c3_instances(seed=0, n=64):
    """64 independent instances: grid in {4x4,5x5,6x6}, chi_max in {16,32,48}, h ~ U[0.5, 3]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        L = int(rng.choice([4, 5, 6]))
        out.append(dict(Lx=L, Ly=L, J=1.0, h=float(rng.uniform(0.5, 3.0)), dt=0.05, order=2,
                        obs=((L - 1) // 2, (L - 1) // 2), chi_max=int(rng.choice([16, 32, 48])),
                        bp_alpha=0.5, bp_tol=1e-5, nsteps=40, precision="fp32"))
    return out
