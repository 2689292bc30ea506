"""Shared test helpers: comparing a GPU hierarchy with an oracle hierarchy; new values on a pattern."""
import numpy as np

import workloads as W


def with_values(s, val, b=None):
    """The system s with new values on its pattern (and optionally a new right-hand side)."""
    return W.CsrSystem(s.n, s.row_ptr.copy(), s.col.copy(), np.asarray(val, np.float64).copy(),
                       s.b.copy() if b is None else b)


def backward_euler(s, dt):
    """I + dt S on S's pattern (S has an explicit diagonal): the time step of Sec. 4.1.1."""
    rows = np.repeat(np.arange(s.n), np.diff(s.row_ptr))
    return with_values(s, dt * s.val + (rows == s.col))


def max_rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.size == 0:
        return 0.0
    scale = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / scale)


def row_rel(rp, a, b):
    """max over rows of max|a - b| / max|b| within the row (inf where a row of b is zero and a differs)"""
    rp = np.asarray(rp, np.int64)
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))
    m = np.abs(np.asarray(b, np.float64))
    lens = np.diff(rp)
    rows = np.nonzero(lens > 0)[0]
    if rows.size == 0:
        return 0.0
    starts = rp[rows]
    dmax = np.maximum.reduceat(d, starts)
    mmax = np.maximum.reduceat(m, starts)
    # reduceat over starts of non-empty rows: each segment runs to the next start, which is this row's end
    if np.any((mmax == 0) & (dmax > 0)):
        return np.inf
    ok = mmax > 0
    return float((dmax[ok] / mmax[ok]).max()) if ok.any() else 0.0


def compare_hierarchies(G, H, val_tol):
    """Integer structure must match bit for bit; values within val_tol (row-relative).
    Returns a dict of the largest value differences seen."""
    ginfo = G.info()
    glev = len(ginfo)
    # the oracle reports a level whose splitting produced no coarse points as a level with cf but no R
    olev = len(H.levels)
    assert glev == olev, f"levels: gpu {glev} oracle {olev} ({[g['n'] for g in ginfo]} vs {[L.n for L in H.levels]})"
    worst = {}
    for l, (gi, L) in enumerate(zip(ginfo, H.levels)):
        rp, col, val = G.export_csr(l, 0)
        assert gi["n"] == L.n, f"level {l}: n {gi['n']} vs {L.n}"
        assert np.array_equal(rp, L.A[0]), f"level {l}: A row pointers differ"
        assert np.array_equal(col, L.A[1]), f"level {l}: A columns differ"
        worst[f"A{l}"] = row_rel(rp, val, L.A[2])
        assert worst[f"A{l}"] <= val_tol, f"level {l}: A values differ by {worst[f'A{l}']:.3e}"
        if gi["coarsest"]:
            break
        cf, strong, lsr, lsp = G.export_cf(l)
        assert np.array_equal(strong, L.strong), f"level {l}: strength masks differ ({(strong != L.strong).sum()})"
        assert np.array_equal(cf, L.cf), f"level {l}: C/F splittings differ ({(cf != L.cf).sum()} points)"
        assert np.array_equal(lsr, L.ls_R), f"level {l}: least-squares flags of R differ"
        if L.ls_P is not None:
            assert np.array_equal(lsp, L.ls_P), f"level {l}: least-squares flags of P differ"
        for which, name, O in ((1, "R", L.R), (2, "P", L.P)):
            rp, col, val = G.export_csr(l, which)
            assert np.array_equal(rp, O[0]), f"level {l}: {name} row pointers differ"
            assert np.array_equal(col, O[1]), f"level {l}: {name} columns differ"
            worst[f"{name}{l}"] = row_rel(rp, val, O[2])
            assert worst[f"{name}{l}"] <= val_tol, f"level {l}: {name} values differ by {worst[f'{name}{l}']:.3e}"
    return worst


def entrywise_rel(z, zo):
    """max over entries of |z - zo| / max |zo| (0 for an empty vector)."""
    z = np.asarray(z, np.float64)
    zo = np.asarray(zo, np.float64)
    if zo.size == 0:
        return 0.0
    return float(np.abs(z - zo).max() / max(np.abs(zo).max(), 1e-300))
