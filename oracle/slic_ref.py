"""Plain numpy reference of the superpixel patch builder, for tests only.

TEST INFRASTRUCTURE ONLY: nothing in the product library imports this file.

Superpixel patches (Sec. II "Patch Extraction", SLIC of the cited work):
per slice, simple linear iterative clustering with initial step a and
compactness t, distance D^2 = d_c^2 + (d_s / a)^2 t^2 (d_c intensity, d_s
spatial distance); each superpixel dilated by gamma pixels with a square
structuring element; a patch is the superpixel's dilated bounding box with a
membership mask.

Readings (the paper leaves them open):
* centres start on a regular grid: nx = max(1, round(W / a)) columns of width
  sx = W / nx (likewise rows), centre (i + 0.5) sx, (j + 0.5) sy, intensity
  the pixel under it;
* a pixel at (x, y) in grid cell (floor(x / sx), floor(y / sy)) (float64,
  clipped) compares the centres of the 3 x 3 neighbouring cells; ties go to
  the lower centre index j * nx + i;
* D^2 is evaluated in float32 as dI*dI + (dx*dx + dy*dy) * m2 with
  m2 = float32((t / a)^2), each operation rounded (no fused multiply-add);
* centres move to the mean position and intensity of their pixels, summed
  exactly in integers (intensities as round(1024 I), half to even) and
  divided in float64, then rounded to float32; a centre without pixels
  stays; n_iter iterations, no connectivity step;
* a superpixel is kept when its dilated box fits max_side and at least
  keep_frac of its member pixels exceed fg_frac * I_max (I_max over all
  stacks);
* table order: stack, slice, centre index; desc {stack, slice, x0, y0, w, h,
  pix_off, 0}; pixel offsets packed over the boxes.
"""
from __future__ import annotations

import numpy as np


def slic_labels(img, a, t, n_iter=10):
    img = np.asarray(img, np.float32)
    H, W = img.shape
    nx, ny = max(1, int(round(W / a))), max(1, int(round(H / a)))
    sx, sy = W / nx, H / ny
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny))
    cx = ((ii + 0.5) * sx).astype(np.float32).reshape(-1)
    cy = ((jj + 0.5) * sy).astype(np.float32).reshape(-1)
    ci = img[np.minimum(cy.astype(np.int64), H - 1), np.minimum(cx.astype(np.int64), W - 1)].astype(np.float32)
    m2 = np.float32((t / a) * (t / a))
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    cellx = np.minimum(np.floor(xx / sx).astype(np.int64), nx - 1)
    celly = np.minimum(np.floor(yy / sy).astype(np.int64), ny - 1)
    xf, yf = xx.astype(np.float32), yy.astype(np.float32)
    labels = np.zeros((H, W), np.int64)
    for _ in range(n_iter):
        best = np.full((H, W), np.inf, np.float32)
        lab = np.zeros((H, W), np.int64)
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                cj, cii = celly + dj, cellx + di
                ok = (cj >= 0) & (cj < ny) & (cii >= 0) & (cii < nx)
                c = np.where(ok, cj * nx + cii, 0)
                dI = img - ci[c]
                dx = xf - cx[c]
                dy = yf - cy[c]
                d = dI * dI + (dx * dx + dy * dy) * m2
                better = ok & ((d < best) | ((d == best) & (c < lab)))
                best = np.where(better, d, best)
                lab = np.where(better, c, lab)
        labels = lab
        K = nx * ny
        cnt = np.bincount(labels.ravel(), minlength=K)
        sxs = np.bincount(labels.ravel(), weights=xx.ravel().astype(np.float64), minlength=K)
        sys_ = np.bincount(labels.ravel(), weights=yy.ravel().astype(np.float64), minlength=K)
        q = np.rint(img.astype(np.float64) * 1024.0).ravel()          # integers, exact in float64
        sis = np.bincount(labels.ravel(), weights=q, minlength=K) / 1024.0
        has = cnt > 0
        cx = np.where(has, (sxs / np.maximum(cnt, 1)).astype(np.float32), cx)
        cy = np.where(has, (sys_ / np.maximum(cnt, 1)).astype(np.float32), cy)
        ci = np.where(has, (sis / np.maximum(cnt, 1)).astype(np.float32), ci)
    return labels, nx * ny


def patches_build_slic(stack_dims, stacks, a, t, gamma, n_iter=10, fg_frac=0.0, keep_frac=0.0, max_side=128):
    """Returns (desc [P, 8] int32, member [n_pix] uint8, n_pix)."""
    stacks = [np.asarray(s, np.float32) for s in stacks]
    imax = max(float(s.max()) for s in stacks)
    thr = np.float32(fg_frac) * np.float32(imax)
    rows, mem, off = [], [], 0
    for si, ((W, H, K), st) in enumerate(zip(stack_dims, stacks)):
        for k in range(K):
            img = st[k]
            labels, nK = slic_labels(img, a, t, n_iter)
            for c in range(nK):
                m = labels == c
                if not m.any():
                    continue
                ys, xs = np.nonzero(m)
                x0, x1 = max(xs.min() - gamma, 0), min(xs.max() + gamma, W - 1)
                y0, y1 = max(ys.min() - gamma, 0), min(ys.max() + gamma, H - 1)
                w, h = x1 - x0 + 1, y1 - y0 + 1
                if w > max_side or h > max_side:
                    continue
                box = m[y0:y1 + 1, x0:x1 + 1]
                dil = np.zeros_like(box)
                for dy in range(-gamma, gamma + 1):
                    for dx in range(-gamma, gamma + 1):
                        src = np.zeros_like(box)
                        ya, yb = max(0, -dy), min(h, h - dy)
                        xa, xb = max(0, -dx), min(w, w - dx)
                        src[ya:yb, xa:xb] = box[ya + dy:yb + dy, xa + dx:xb + dx]
                        dil |= src
                n_mem = int(dil.sum())
                fg = int((img[y0:y1 + 1, x0:x1 + 1][dil] > thr).sum())
                if not (fg >= keep_frac * n_mem):
                    continue
                rows.append([si, k, x0, y0, w, h, off, 0])
                mem.append(dil.astype(np.uint8).reshape(-1))
                off += w * h
    desc = np.array(rows, np.int32).reshape(-1, 8)
    member = np.concatenate(mem) if mem else np.zeros(0, np.uint8)
    return desc, member, off
