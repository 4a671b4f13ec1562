"""Oracle: bucket elimination with explicit slicing, in complex128 (Alg. 1, Eq. 2).

TEST INFRASTRUCTURE (see oracle/network.py).

Bucket elimination (Alg. 1): with the order pi, bucket B_i holds the tensors
whose earliest index with respect to pi is pi^-1(i). Processing the buckets in
order, the tensors of a bucket are multiplied over the union of their indices
and the bucket's variable is summed out; a scalar result multiplies the
running result, any other result goes to the bucket of its earliest index.

Slicing (Alg. 1, Eq. 2): after the first s buckets have been processed on the
unsliced network (contract_first), every sliced index is fixed to one value in
every remaining tensor, the remaining buckets are processed per slice, and the
slice results are summed (the paper's final reduce-sum), here in slice-id
order. Slice id bit j is the value of the j-th sliced variable.
"""

from __future__ import annotations

import numpy as np


def _einsum_product_sum(operands, out_labels):
    """Product of all operands over the union of their labels, summed to out_labels."""
    letters = {}
    args = []
    for labels, data in operands:
        args.append(data)
        args.append([letters.setdefault(l, len(letters)) for l in labels])
    if len(letters) > 52:
        raise ValueError("too many indices for einsum")
    args.append([letters[l] for l in out_labels])
    return np.einsum(*args, optimize=False)


def _earliest(labels, pos):
    ranked = [pos[l] for l in labels if l in pos]
    return min(ranked) if ranked else None


def eliminate_buckets(tensors, order, pos):
    """Process the buckets of the variables in `order` (positions from `pos`).

    Returns (scalar, remaining): the product of the scalar results and the
    tensors left once those buckets are gone (tensors whose labels have no
    position in `order` stay untouched).
    """
    first = {v: i for i, v in enumerate(order)}
    buckets = [[] for _ in order]
    remaining = []
    scalar = complex(1.0)

    def place(t):
        nonlocal scalar
        labels, data = t
        if len(labels) == 0:
            scalar *= complex(data)
            return
        e = _earliest(labels, pos)
        v = None
        if e is not None:
            v = next(l for l in labels if pos.get(l) == e)
        if v is not None and v in first:
            buckets[first[v]].append(t)
        else:
            remaining.append(t)

    for t in tensors:
        place(t)
    for i, v in enumerate(order):
        bucket = buckets[i]
        if not bucket:
            continue
        union = []
        for labels, _ in bucket:
            for l in labels:
                if l not in union:
                    union.append(l)
        out = sorted((l for l in union if l != v), key=lambda l: (pos.get(l, 1 << 40), l))
        res = _einsum_product_sum(bucket, out)
        place((tuple(out), np.asarray(res)))
    return scalar, remaining


def fix_indices(tensors, values):
    """Slice every tensor: index l takes the value values[l] for each l in values."""
    out = []
    for labels, data in tensors:
        idx = tuple(values[l] if l in values else slice(None) for l in labels)
        new_labels = tuple(l for l in labels if l not in values)
        out.append((new_labels, np.asarray(data[idx])))
    return out


def _finish(scalar, rest, open_vars):
    """Product of the scalar and the tensors left over the open variables (outer
    product into a tensor with axis j = open_vars[j]); a scalar when none is open."""
    if not open_vars:
        if rest:
            raise ValueError("variables left uneliminated")
        return scalar
    for labels, _ in rest:
        if not set(labels) <= set(open_vars):
            raise ValueError("variables left uneliminated")
    out = _einsum_product_sum(rest, list(open_vars)) if rest else np.ones((2,) * len(open_vars))
    return scalar * np.asarray(out)


def contract_amplitude(tensors, order, sliced=(), slice_step=0, slice_ids=None, open_vars=()):
    """Full contraction of the network along `order` with the given slicing.

    Returns (total, per_slice): total is the sum of the slice results over
    slice_ids (all 2^k ids when None) and per_slice the list of those results.
    Without sliced variables there is one slice and slice_step is ignored. With
    open variables (a batch of amplitudes, Sec. VII) the results are tensors over
    them (axis j = open_vars[j]).
    """
    sliced = list(sliced)
    k = len(sliced)
    pos = {v: i for i, v in enumerate(order)}
    if k == 0:
        s, rest = eliminate_buckets(tensors, list(order), pos)
        res = _finish(s, rest, open_vars)
        return res, [res]
    prefix = list(order[:slice_step])
    suffix = list(order[slice_step:])
    pre_scalar, remaining = eliminate_buckets(tensors, prefix, pos)
    if slice_ids is None:
        slice_ids = range(1 << k)
    per_slice = []
    total = 0
    for sid in slice_ids:
        values = {v: (sid >> j) & 1 for j, v in enumerate(sliced)}
        part = fix_indices(remaining, values)
        s, rest = eliminate_buckets(part, suffix, pos)
        res = pre_scalar * _finish(s, rest, open_vars)
        per_slice.append(res)
        total = total + res
    return total, per_slice
