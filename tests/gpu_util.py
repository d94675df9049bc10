"""Helpers shared by the GPU parity tests (upload/download of heap contents)."""
import numpy as np
import torch


def upload(heap, init: np.ndarray):
    heap.partitions().copy_(torch.from_numpy(init.reshape(heap.npes, heap.H)).cuda())


def download(heap) -> np.ndarray:
    torch.cuda.synchronize()
    return heap.partitions().cpu().numpy().reshape(-1)


def random_heap(npes, H, seed):
    import workloads as W

    return W.cb64_np(seed, np.arange(npes * H // 8, dtype=np.uint64)).view(np.uint8).copy()


def first_diff(a, b):
    d = np.nonzero(a != b)[0]
    return None if len(d) == 0 else (int(d[0]), len(d))
