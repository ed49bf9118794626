"""Low-storage fourth-order Runge-Kutta time stepping (oracle).

Test infrastructure only; see ``oracle/__init__.py``.

The paper integrates in time with the five-stage, two-register (2N-storage)
fourth-order scheme of Carpenter & Kennedy (1994), cited in Sections 1 and 7
without its coefficients.  The coefficients below are the published (5,4)
2N-storage solution; they are checked by tests against the classical order
conditions and by an observed-order test, not trusted.

One step from (Q, t) with step dt, for stages k = 0..4:
    dQ <- A_k dQ + dt * L(Q, t + c_k dt)
    Q  <- Q + B_k dQ
"""
from fractions import Fraction as Fr

RK_A = (Fr(0), Fr(-567301805773, 1357537059087), Fr(-2404267990393, 2016746695238),
        Fr(-3550918686646, 2091501179385), Fr(-1275806237668, 842570457699))
RK_B = (Fr(1432997174477, 9575080441755), Fr(5161836677717, 13612068292357),
        Fr(1720146321549, 2090206949498), Fr(3134564353537, 4481467310338),
        Fr(2277821191437, 14882151754819))


def _stage_times():
    """c_k = sum_j a_kj of the equivalent Butcher tableau (consistency of the stage times).

    Stage k evaluates L at Q_0 + sum_{m<k} B_m dQ_m, and dQ_m collects dt f_j with
    weight prod A over the stages between j and m; c_k is the total weight.
    The stage times are derived here rather than quoted because a quoted rational
    for c_2 disagreed with A and B in the eighth digit.
    """
    c = []
    reg = [Fr(0)] * 5          # weight of dt f_j in the register
    acc = [Fr(0)] * 5          # weight of dt f_j in Q
    for k in range(5):
        c.append(sum(acc))
        reg = [RK_A[k] * reg[j] + (1 if j == k else 0) for j in range(5)]
        acc = [acc[j] + RK_B[k] * reg[j] for j in range(5)]
    return tuple(c)


RK_C = _stage_times()

A = tuple(float(x) for x in RK_A)
B = tuple(float(x) for x in RK_B)
C = tuple(float(x) for x in RK_C)


def rk_step(Q, dQ, t, dt, L):
    """Advance (Q, dQ) one step in place.  ``L(Q, t)`` returns dQ/dt (same shape)."""
    for k in range(5):
        dQ *= A[k]
        dQ += dt * L(Q, t + C[k] * dt)
        Q += B[k] * dQ
    return Q, dQ


def butcher_tableau():
    """Equivalent Butcher tableau (a_ij, b_i, c_i) of the 2N-storage scheme, as Fractions.

    With register recursion dQ_k = A_k dQ_{k-1} + dt f_k and Q_k = Q_{k-1} + B_k dQ_k,
    stage k sees Q_{k-1} = Q_0 + sum_{j<k} a_kj dt f_j.
    """
    s = 5
    # coefficient of dt f_j in dQ_k
    reg = [[Fr(0)] * s for _ in range(s)]
    a = [[Fr(0)] * s for _ in range(s)]
    acc = [Fr(0)] * s            # coefficient of dt f_j in Q_k - Q_0
    for k in range(s):
        for j in range(s):
            reg[k][j] = (RK_A[k] * reg[k - 1][j] if k > 0 else Fr(0)) + (1 if j == k else 0)
        a[k] = list(acc)
        acc = [acc[j] + RK_B[k] * reg[k][j] for j in range(s)]
    return a, acc, [sum(row) for row in a]
