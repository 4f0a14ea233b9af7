"""Writes the post-shock water state used by the shock workloads.

TEST INFRASTRUCTURE ONLY.  Run ``python -m oracle.shock_constants`` to print the
density, velocity and shock speed of water (gamma=4.4, pinf=6e8 Pa, rho=1000,
p=1e5, at rest) behind a shock to p=1e9 Pa; ``workloads.py`` stores these
numbers and a CPU test checks them against this computation.
"""
from oracle.exact_riemann import Side, shocked_state


def post_shock_water(p_post: float = 1.0e9):
    return shocked_state(Side(1000.0, 0.0, 1.0e5, 4.4, 6.0e8), p_post)


if __name__ == "__main__":
    rho, u, s = post_shock_water()
    print("SHOCK_RHO = %r\nSHOCK_U = %r\nSHOCK_SPEED = %r" % (rho, u, s))
