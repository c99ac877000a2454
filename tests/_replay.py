"""Decision traces of the GPU's adaptive Krylov evaluations, split per
evaluation, in the form the oracle replays (the arithmetic is the oracle's;
only the substep sizes and basis sizes are taken from the GPU run)."""


def forced(trace):
    """One evaluation's (tau, m) list as the oracle's forced trace."""
    return [(t, m, 0) for t, m in trace]


def split_evaluations(trace, n_eval):
    """A step's trace lists the substeps of its n_eval evaluations in order;
    each evaluation's substeps end where their steps add up to 1."""
    out, cur, t = [], [], 0.0
    for tau, m in trace:
        cur.append((tau, m, 0))
        t += tau
        if t >= 1.0 - 1e-9:
            out.append(cur)
            cur, t = [], 0.0
    assert not cur and len(out) == n_eval, (trace, n_eval)
    return out
