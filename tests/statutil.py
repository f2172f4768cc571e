"""Error bars for Markov-chain averages in the tests: blocking into equal
sub-ensembles (section IV.B of Hasenbusch & Schaefer quotes errors from ten
blocks)."""
import numpy as np


def block_mean_err(x, n_blocks=20, axis=0):
    """Mean and blocking error of x along `axis` (drops the ragged tail)."""
    x = np.moveaxis(np.asarray(x, float), axis, 0)
    n = (x.shape[0] // n_blocks) * n_blocks
    b = x[:n].reshape(n_blocks, n // n_blocks, *x.shape[1:]).mean(1)
    return b.mean(0), b.std(0, ddof=1) / np.sqrt(n_blocks)


def within(a, ea, b, eb, nsig=4.0):
    """Boolean array: |a - b| <= nsig * sqrt(ea^2 + eb^2)."""
    return np.abs(np.asarray(a) - np.asarray(b)) <= nsig * np.sqrt(np.asarray(ea) ** 2 + np.asarray(eb) ** 2)
