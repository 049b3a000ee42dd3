"""Helpers shared by the tests."""
import numpy as np


def rel_err(got, want, floor=1e-6):
    """max_i |g_i - o_i| / max(|o_i|, floor * max|o|): the parity measure of the year map."""
    got = np.asarray(got)
    want = np.asarray(want)
    scale = np.maximum(np.abs(want), floor * np.abs(want).max())
    return float(np.max(np.abs(got - want) / scale))


def normwise_err(got, want):
    """max_i |g_i - o_i| / max_i |o_i|: the measure for signed fields (tangents, cotangents),
    whose elements pass through zero, so that a relative error per element is not defined."""
    got = np.asarray(got)
    want = np.asarray(want)
    return float(np.max(np.abs(got - want)) / np.max(np.abs(want)))
