"""A free-running FP64 oracle trajectory in a child process (test infrastructure).

Long GPU runs compare their states with the oracle every few steps; the oracle's
own steps are slow, so it runs beside the GPU loop in a process started with the
'spawn' method (never forked from a process that has touched the GPU).  The
child imports only numpy and the oracle.

Protocol over a multiprocessing Pipe: the parent sends (t, Xt) for every step t
(Xt: (n, d) float64, the batch the GPU received) and None to finish; the child
applies oracle.init (t == 0) or oracle.update, and after every step t with
(t + 1) % every == 0 sends back (t, Ut, sigma) of the current rank.
"""
import os
import sys


def run(conn, root, r, rho, every, threads):
    if root not in sys.path:
        sys.path.insert(0, root)
    import oracle

    oracle.build()
    oracle.set_threads(threads)
    U = s = None
    k = 0
    while True:
        msg = conn.recv()
        if msg is None:
            break
        t, X = msg
        if t == 0:
            U, s, info = oracle.init(X, r)
        else:
            U, s, info = oracle.update(U[:k], s[:k], k, X, rho, r)
        k = info["r_new"]
        if (t + 1) % every == 0:
            conn.send((t, U[:k].copy(), s[:k].copy()))
    conn.close()


def start(r, rho, every, threads):
    """Starts a worker; returns (process, parent end of the pipe)."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    parent, child = ctx.Pipe()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    p = ctx.Process(target=run, args=(child, root, r, rho, every, threads), daemon=True)
    p.start()
    child.close()
    return p, parent
