"""Test-side conversions between the oracle's (m, e) pairs and the library's
(sign, exp, limbs) arrays, and torch device staging for the primitives."""
import numpy as np

from oracle import mpfloat as F


def to_arrays(nums, n):
    cnt = len(nums)
    s = np.zeros(cnt, np.int32)
    e = np.zeros(cnt, np.int32)
    m = np.zeros((cnt, n), np.uint32)
    for i, x in enumerate(nums):
        sg, ex, limbs = F.limbs_of(x, n)
        s[i], e[i] = sg, ex
        m[i] = limbs
    return s, e, m


def from_arrays(s, e, m):
    return [F.from_limbs(int(s[i]), int(e[i]), m[i]) for i in range(len(s))]


class DevNums:
    """count numbers of n limbs on the current CUDA device (torch-owned)."""

    def __init__(self, nums=None, count=None, n=None):
        import torch
        if nums is not None:
            s, e, m = to_arrays(nums, n)
        else:
            s = np.zeros(count, np.int32)
            e = np.zeros(count, np.int32)
            m = np.zeros((count, n), np.uint32)
        self.n = n
        self.s = torch.from_numpy(s).cuda()
        self.e = torch.from_numpy(e).cuda()
        self.m = torch.from_numpy(m.view(np.int32)).cuda()

    @property
    def ptrs(self):
        return (self.s.data_ptr(), self.e.data_ptr(), self.m.data_ptr())

    def to_host(self):
        return from_arrays(self.s.cpu().numpy(), self.e.cpu().numpy(), self.m.cpu().numpy().view(np.uint32))
