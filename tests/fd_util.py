"""Central finite differences of the loss L(u0) = dtau sum u_end^2 for the
adjoint tests (oracle on the CPU, CUDA path on the GPU).

The loss difference L(x+) - L(x-) is summed as dtau sum (y+ - y-)(y+ + y-),
an exact factorisation of y+^2 - y-^2: the difference of two sums of squares
would cancel about half of the FP64 digits before the division by 2h.  The
perturbation actually applied is x+ - x- with x+- = fl(u0 +- h v); the
adjoint's directional derivative is taken along that vector, so the rounding
of u0 + h v is the same on both sides of the comparison.
"""


def central_fd_numpy(advance, u0, v, h, dtau, g0):
    """(ad, fd): <g0, (x+ - x-)/(2h)> and the central difference of the loss,
    ``advance(x)`` returning the state after the steps (numpy FP64)."""
    import numpy as np
    xp, xm = u0 + h * v, u0 - h * v
    yp, ym = advance(xp), advance(xm)
    fd = float(np.sum((yp - ym) * (yp + ym))) * dtau / (2 * h)
    ad = float(np.sum(g0 * (xp - xm))) / (2 * h)
    return ad, fd


def central_fd_torch(plan, u0, v, h, n_steps, dtau, g0, sigma0=0.0):
    """(ad, fd) for a CUDA plan: u0, v, g0 device tensors of the plan's shape."""
    xp, xm = u0 + h * v, u0 - h * v
    yp, ym = xp.clone(), xm.clone()
    plan.advance(yp, n_steps, sigma0=sigma0)
    plan.advance(ym, n_steps, sigma0=sigma0)
    fd = float(((yp - ym) * (yp + ym)).sum()) * dtau / (2 * h)
    ad = float((g0 * (xp - xm)).sum()) / (2 * h)
    return ad, fd


def fd_bound(tol, fd, g0_norm, n_points):
    """Allowed |ad - fd|: tol * max(|fd|, 0.1 |g0| / sqrt(N)).

    For a random unit direction v, <g0, v> has standard deviation
    |g0| / sqrt(N).  The central difference carries a rounding floor that does
    not depend on v (the forward runs' own rounding, divided by 2h), so in the
    rare direction whose derivative falls below a tenth of that scale (about
    8 % of Gaussian directions) the comparison is made at a tenth of the scale
    instead of at |fd|; everywhere else it is relative to |fd|."""
    return tol * max(abs(fd), 0.1 * g0_norm / n_points ** 0.5)
