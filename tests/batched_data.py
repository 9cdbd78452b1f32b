"""Inputs of the batched triples workload T[a,b,c,i,j,k] = sum_d A[d,a,b,i] * B[c,d,j,k]:
per-block operands packed into one device buffer per operand kind, seeded normal(0, 0.1)."""
import numpy as np

import synth

EXPR = "T[a,b,c,i,j,k] = A[d,a,b,i] * B[c,d,j,k]"
LABELS = ["a", "b", "c", "i", "j", "k", "d"]


def shapes(ext_row):
    a, b, c, i, j, k, d = [int(x) for x in ext_row]
    return (d, a, b, i), (c, d, j, k), (a, b, c, i, j, k)


class Blocks:
    def __init__(self, ext, dtype, device="cuda", seed=3, exact_blocks=()):
        import torch
        self.ext = np.asarray(ext, dtype=np.int64)
        self.n = len(self.ext)
        self.tdt = torch.float32 if dtype == np.float32 else torch.float64
        self.np_dtype = dtype
        align = 4 if dtype == np.float32 else 2
        offs = [[0, 0] for _ in range(self.n)]
        tot = [0, 0]
        for b in range(self.n):
            sa, sb, _ = shapes(self.ext[b])
            for o, s in enumerate((sa, sb)):
                offs[b][o] = tot[o]
                tot[o] += (int(np.prod(s)) + align - 1) // align * align
        self.offs, self.tot = offs, tot
        self.buf = [synth.torch_normal(seed, o, tot[o], device, dtype=self.tdt, std=0.1) for o in range(2)]
        # blocks the oracle will see: their values come from the host generator, so both sides
        # read identical inputs
        for b in exact_blocks:
            for o in range(2):
                v = self.host_operand(b, o)
                self.buf[o][offs[b][o]:offs[b][o] + v.size] = torch.from_numpy(
                    np.ascontiguousarray(np.ravel(v, order="F"))).to(device)
        ptrs = []
        es = 4 if dtype == np.float32 else 8
        for b in range(self.n):
            for o in range(2):
                ptrs.append(self.buf[o].data_ptr() + es * offs[b][o])
        self.ptrs = torch.tensor(ptrs, dtype=torch.int64, device=device)

    def host_operand(self, b, o, seed=3):
        s = shapes(self.ext[b])[o]
        n = int(np.prod(s))
        v = synth.normal_range(seed, o, self.offs[b][o], n, std=0.1).astype(self.np_dtype)
        return np.asfortranarray(v.reshape(s, order="F"))

    def flops(self, b):
        return 2.0 * float(np.prod(self.ext[b]))
