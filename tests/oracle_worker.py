"""A free-running FP64 oracle trajectory in a child process (test infrastructure).

Long GPU runs compare their states with the oracle every few steps; the oracle's
own steps are slow, so it runs beside the GPU loop in a process started with the
'spawn' method (never forked from a process that has touched the GPU).  The
child imports only numpy and the oracle.

Protocol over two one-way pipes: the parent sends (t, Xt) for every step t
(Xt: (n, d) float64, the batch the GPU received) and None to finish; the child
applies the oracle's update (from k = 0 with rho = 0 for t == 0, the exact first
state; oracle.update_eigh, the update with LAPACK's eigensolver for the core,
pinned to the Jacobi oracle), and after every step t with (t + 1) % every == 0
sends back (t, Ut, sigma) of the current rank, then None when done.  A thread of
the parent drains the results while its main thread sends batches, so neither
side ever blocks on a full pipe.
"""
import os
import sys


def run(rx, tx, root, r, rho, every, threads):
    if root not in sys.path:
        sys.path.insert(0, root)
    import numpy as np

    import oracle

    oracle.build()
    oracle.set_threads(threads)
    U = s = None
    k = 0
    while True:
        msg = rx.recv()
        if msg is None:
            break
        t, X = msg
        if t == 0:
            U, s, info = oracle.update_eigh(np.zeros((1, X.shape[1])), np.zeros(1), 0, X, 0.0, r)
        else:
            U, s, info = oracle.update_eigh(U[:k], s[:k], k, X, rho, r)
        k = info["r_new"]
        if (t + 1) % every == 0:
            tx.send((t, U[:k].copy(), s[:k].copy()))
    tx.send(None)
    tx.close()


class Worker:
    """A spawned oracle trajectory: send(t, X) each step, finish() -> [(t, Ut, sigma)]."""

    def __init__(self, r, rho, every, threads):
        import multiprocessing as mp
        import threading

        ctx = mp.get_context("spawn")
        rx_child, self._tx = ctx.Pipe(duplex=False)   # parent -> child batches
        self._rx, tx_child = ctx.Pipe(duplex=False)   # child -> parent results
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        self.proc = ctx.Process(target=run, args=(rx_child, tx_child, root, r, rho, every, threads), daemon=True)
        # the child inherits the environment: one BLAS thread (its eigensolves are small)
        # and `threads` OpenMP threads for the oracle's loops, so that workers running
        # side by side do not oversubscribe the cores
        keys = ("OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "OMP_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        os.environ.update({"OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1", "OMP_NUM_THREADS": str(threads)})
        try:
            self.proc.start()
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        rx_child.close()
        tx_child.close()
        self.results = []
        self.error = None

        def drain():
            try:
                while True:
                    m = self._rx.recv()
                    if m is None:
                        break
                    self.results.append(m)
            except (EOFError, OSError) as e:
                self.error = e

        self._thread = threading.Thread(target=drain, daemon=True)
        self._thread.start()

    def send(self, t, X):
        self._tx.send((t, X))

    def finish(self, timeout=600):
        self._tx.send(None)
        self._thread.join(timeout)
        self.proc.join(timeout=60)
        if self.proc.is_alive():
            self.proc.kill()
        if self._thread.is_alive() or self.error is not None:
            raise RuntimeError(f"oracle worker did not finish: {self.error}")
        return self.results

    def kill(self):
        if self.proc.is_alive():
            self.proc.kill()
