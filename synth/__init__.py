"""Seeded synthetic inputs for the reprojection path: sky images and TAN(-SIP) WCS records.

This module is shared by the tests, the oracle checks and the benchmark. It holds no
reprojection arithmetic: it only draws random numbers and formats them as images, WCS
parameter records and FITS header cards.

Inputs stand in for the paper's Dragonfly exposures and its 50x50 demo files (Sec. 2, Sec. 4),
which are not available; sizes span the paper's 256x256 to 4000x6000 range (Sec. 4.2).

WCS record (a plain dict, the same fields as the C ``dfr_wcs`` struct):
    naxis  (W, H)                 NAXIS1 (x, fastest axis), NAXIS2
    crpix  (c1, c2)               FITS 1-based reference pixel
    crval  (ra0, dec0)            degrees
    cd     2x2 nested list        degrees / pixel
    a_order, b_order, ap_order, bp_order   0 = absent
    a, b, ap, bp                  10x10 float64 arrays, [p][q] = coefficient of u^p v^q
"""
from __future__ import annotations

import math

import numpy as np

MAX_SIP = 9
FWHM_PX = 3.0
SIGMA_PX = FWHM_PX / (2.0 * math.sqrt(2.0 * math.log(2.0)))


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------- WCS records
def empty_sip() -> np.ndarray:
    return np.zeros((MAX_SIP + 1, MAX_SIP + 1), dtype=np.float64)


def cd_matrix(scale_deg: float, rho_deg: float) -> list:
    """CD from CDELT1 = -s, CDELT2 = +s and a CROTA2-style rotation rho (degrees)."""
    c, s = math.cos(math.radians(rho_deg)), math.sin(math.radians(rho_deg))
    return [[-scale_deg * c, -scale_deg * s], [-scale_deg * s, scale_deg * c]]


def tan_wcs(width: int, height: int, crval=(150.0, 2.0), scale_arcsec=2.5, rho_deg=0.0,
            crpix=None) -> dict:
    if crpix is None:
        crpix = ((width + 1) / 2.0, (height + 1) / 2.0)
    return {
        "naxis": (int(width), int(height)),
        "crpix": (float(crpix[0]), float(crpix[1])),
        "crval": (float(crval[0]), float(crval[1])),
        "cd": cd_matrix(scale_arcsec / 3600.0, rho_deg),
        "a_order": 0, "b_order": 0, "ap_order": 0, "bp_order": 0,
        "a": empty_sip(), "b": empty_sip(), "ap": empty_sip(), "bp": empty_sip(),
    }


def copy_wcs(w: dict) -> dict:
    out = dict(w)
    out["cd"] = [list(w["cd"][0]), list(w["cd"][1])]
    for k in ("a", "b", "ap", "bp"):
        out[k] = np.array(w[k], dtype=np.float64, copy=True)
    return out


def sip_terms(order: int):
    """(p, q) with 1 <= p+q <= order, ordered by p+q then p descending."""
    out = []
    for n in range(1, order + 1):
        for p in range(n, -1, -1):
            out.append((p, n - p))
    return out


def draw_sip(order: int, sigma0: float, radius_px: float, rng: np.random.Generator):
    """Forward SIP A, B with sigma_pq = sigma0 * R^(2-(p+q)) for 2 <= p+q <= order.

    Linear terms are zero. With this scaling each term moves a frame corner by about
    sigma0 * R^2 pixels, which keeps the distortion invertible for sigma0 = 1e-6 / 1e-7.
    """
    a, b = empty_sip(), empty_sip()
    for (p, q) in sip_terms(order):
        if p + q < 2:
            continue
        sig = sigma0 * radius_px ** (2 - (p + q))
        a[p, q] = rng.normal(0.0, sig)
        b[p, q] = rng.normal(0.0, sig)
    return a, b


def add_sip(w: dict, order: int, sigma0: float, rng: np.random.Generator) -> dict:
    w = copy_wcs(w)
    radius = max(w["naxis"]) / 2.0
    a, b = draw_sip(order, sigma0, radius, rng)
    w["a"], w["b"] = a, b
    w["a_order"] = w["b_order"] = order
    return w


# ----------------------------------------------------------------------------- images
def sky_image(width: int, height: int, n_sources: int, rng: np.random.Generator,
              noise_sigma: float = 1.0) -> np.ndarray:
    """N(0, 1) sky noise plus Gaussian point sources (FWHM 3 px, peak ~ lognormal(3, 1)).

    Positions are uniform over [0, W) x [0, H). Each source is rendered on an 11x11 stamp.
    """
    img = rng.standard_normal((height, width), dtype=np.float32)
    if noise_sigma != 1.0:
        img *= np.float32(noise_sigma)
    xs = rng.uniform(0.0, width, n_sources)
    ys = rng.uniform(0.0, height, n_sources)
    amp = rng.lognormal(3.0, 1.0, n_sources)
    half = 5
    inv2s2 = 1.0 / (2.0 * SIGMA_PX * SIGMA_PX)
    for x, y, a in zip(xs, ys, amp):
        ix, iy = int(round(x)), int(round(y))
        x0, x1 = max(ix - half, 0), min(ix + half + 1, width)
        y0, y1 = max(iy - half, 0), min(iy + half + 1, height)
        if x0 >= x1 or y0 >= y1:
            continue
        gx = np.exp(-((np.arange(x0, x1) - x) ** 2) * inv2s2)
        gy = np.exp(-((np.arange(y0, y1) - y) ** 2) * inv2s2)
        img[y0:y1, x0:x1] += (a * np.outer(gy, gx)).astype(np.float32)
    return img


def sources_for_area(width: int, height: int, per_16mpix: int = 2000) -> int:
    return max(1, int(round(per_16mpix * width * height / (4096.0 * 4096.0))))


# ----------------------------------------------------------------------------- FITS cards
def _card(key: str, value) -> str:
    if isinstance(value, str):
        v = "'%-8s'" % value
    elif isinstance(value, (int, np.integer)):
        v = "%20d" % int(value)
    else:
        v = "%20s" % repr(float(value)).upper().replace("E", "E")
    s = "%-8s= %s" % (key, v)
    return s[:80].ljust(80)


def header_cards(w: dict, sep: str = "") -> str:
    """Format a WCS record as FITS header cards (80-char records, optional separator)."""
    sip = w["a_order"] > 0 or w["b_order"] > 0
    cards = [
        "SIMPLE  =                    T".ljust(80),
        _card("BITPIX", -32),
        _card("NAXIS", 2),
        _card("NAXIS1", w["naxis"][0]),
        _card("NAXIS2", w["naxis"][1]),
        _card("CTYPE1", "RA---TAN-SIP" if sip else "RA---TAN"),
        _card("CTYPE2", "DEC--TAN-SIP" if sip else "DEC--TAN"),
        _card("CRPIX1", w["crpix"][0]),
        _card("CRPIX2", w["crpix"][1]),
        _card("CRVAL1", w["crval"][0]),
        _card("CRVAL2", w["crval"][1]),
        _card("CD1_1", w["cd"][0][0]),
        _card("CD1_2", w["cd"][0][1]),
        _card("CD2_1", w["cd"][1][0]),
        _card("CD2_2", w["cd"][1][1]),
    ]
    for name in ("a", "b", "ap", "bp"):
        order = w[name + "_order"]
        if order <= 0:
            continue
        cards.append(_card(name.upper() + "_ORDER", order))
        c = w[name]
        for p in range(order + 1):
            for q in range(order + 1 - p):
                if c[p, q] != 0.0:
                    cards.append(_card("%s_%d_%d" % (name.upper(), p, q), c[p, q]))
    cards.append("END".ljust(80))
    return sep.join(cards)


# ----------------------------------------------------------------------------- workloads
def config0(seed: int = 1000) -> dict:
    """512x512 TAN source, no SIP; target shifted (3.7, -2.2) px and rotated 0.5 deg; bilinear."""
    rng = rng_for(seed)
    src = tan_wcs(512, 512)
    tgt = tan_wcs(512, 512, rho_deg=0.5,
                  crpix=(src["crpix"][0] + 3.7, src["crpix"][1] - 2.2))
    img = sky_image(512, 512, 50, rng)
    return {"name": "tan512_bilinear", "src": [src], "tgt": tgt, "images": [img],
            "order": "bilinear", "inverse_order": 0}


def config1(seed: int = 1001) -> dict:
    """4096x4096 TAN-SIP order 3 (sigma0 1e-6), target rotated 1.2 deg, offset (41.3, -17.9),
    1% larger pixel scale; bicubic. AP/BP (order 4) are fitted by the caller."""
    rng = rng_for(seed)
    src = add_sip(tan_wcs(4096, 4096), 3, 1e-6, rng)
    tgt = tan_wcs(4096, 4096, scale_arcsec=2.5 * 1.01, rho_deg=1.2,
                  crpix=(src["crpix"][0] + 41.3, src["crpix"][1] - 17.9))
    img = sky_image(4096, 4096, 2000, rng)
    return {"name": "sip3_4096_bicubic", "src": [src], "tgt": tgt, "images": [img],
            "order": "bicubic", "inverse_order": 4}


def _dithered_frames(n, rng, side_range, aspect_range, dither, rot_max, order, sigma0,
                     fixed_shape=None):
    frames = []
    for _ in range(n):
        if fixed_shape is None:
            long_side = int(rng.integers(side_range[0], side_range[1] + 1))
            aspect = rng.uniform(*aspect_range)
            short = int(round(long_side / aspect))
            w_, h_ = long_side, short
        else:
            w_, h_ = fixed_shape
        dx, dy = rng.uniform(-dither, dither, 2)
        rho = rng.uniform(-rot_max, rot_max)
        w = tan_wcs(w_, h_, rho_deg=rho, crpix=((w_ + 1) / 2.0 + dx, (h_ + 1) / 2.0 + dy))
        w = add_sip(w, order, sigma0, rng)
        frames.append(w)
    return frames


def config2(seed: int = 1002, n_frames: int = 64, with_images: bool = True) -> dict:
    """64 exposures, long side U[2048, 6144], aspect U[1, 1.5], SIP 3, dithers +-50 px,
    rotations +-2 deg, onto one 8192x8192 TAN target; bilinear; per-frame footprints."""
    rng = rng_for(seed)
    frames = _dithered_frames(n_frames, rng, (2048, 6144), (1.0, 1.5), 50.0, 2.0, 3, 1e-6)
    tgt = tan_wcs(8192, 8192, crpix=(4096.5, 4096.5))
    imgs = None
    if with_images:
        imgs = [sky_image(f["naxis"][0], f["naxis"][1],
                          sources_for_area(*f["naxis"]), rng) for f in frames]
    return {"name": "batch64_sip3_8192_bilinear", "src": frames, "tgt": tgt,
            "images": imgs, "order": "bilinear", "inverse_order": 4}


def config3(seed: int = 1003) -> dict:
    """2048x2048 TAN-SIP order 3 for differentiation; target = TAN part, same size; bilinear.

    The perturbed copy adds 0.3 arcsec to both CRVAL, scales CD by (1 + 1e-4) and A/B by 1.1.
    """
    rng = rng_for(seed)
    src = add_sip(tan_wcs(2048, 2048), 3, 1e-6, rng)
    tgt = tan_wcs(2048, 2048)
    img = sky_image(2048, 2048, 500, rng)
    pert = copy_wcs(src)
    pert["crval"] = (src["crval"][0] + 0.3 / 3600.0, src["crval"][1] + 0.3 / 3600.0)
    pert["cd"] = [[c * (1.0 + 1e-4) for c in row] for row in src["cd"]]
    pert["a"] = src["a"] * 1.1
    pert["b"] = src["b"] * 1.1
    return {"name": "grad_sip3_2048_bilinear", "src": [src], "tgt": tgt, "images": [img],
            "order": "bilinear", "inverse_order": 4, "perturbed": pert}


def config4(seed: int = 1004, n_frames: int = 32, with_images: bool = True) -> dict:
    """32 exposures of 6000x4000, SIP order 5 (sigma0 1e-7), dithers +-200 px, rotations +-3 deg,
    bicubic onto a 12000x8000 TAN target; AP/BP order 6."""
    rng = rng_for(seed)
    frames = _dithered_frames(n_frames, rng, None, None, 200.0, 3.0, 5, 1e-7,
                              fixed_shape=(6000, 4000))
    tgt = tan_wcs(12000, 8000, crpix=(6000.5, 4000.5))
    imgs = None
    if with_images:
        imgs = [sky_image(6000, 4000, sources_for_area(6000, 4000), rng) for _ in frames]
    return {"name": "stack32_sip5_12000x8000_bicubic", "src": frames, "tgt": tgt,
            "images": imgs, "order": "bicubic", "inverse_order": 6}


def demo50(seed: int = 1050) -> dict:
    """50x50 pair: target CRPIX moved by half a pixel and CRVAL2 by 0.005 deg (Sec. 4.1); bilinear."""
    rng = rng_for(seed)
    src = tan_wcs(50, 50)
    tgt = tan_wcs(50, 50, crval=(150.0, 2.005),
                  crpix=(src["crpix"][0] + 0.5, src["crpix"][1] + 0.5))
    img = sky_image(50, 50, 3, rng)
    return {"name": "demo50_bilinear", "src": [src], "tgt": tgt, "images": [img],
            "order": "bilinear", "inverse_order": 0}


ORDERS = {"nearest": 0, "bilinear": 1, "bicubic": 2}
