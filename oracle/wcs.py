"""Oracle WCS transforms in FP64 (TEST INFRASTRUCTURE: only tests, smoke() and the bench's
CPU-baseline leg may use this module).

Follows dfreproject Sec. 3.1 and Sec. 3.2 step by step, in the paper's notation:

    Sec. 3.2.1 (target WCS, pixel -> world)
        u = x - (crpix1 - 1), v = y - (crpix2 - 1)
        SIP A/B distortion of (u, v)
        (u', v') = CD (u, v)                          [degrees]
        r = sqrt(u'^2 + v'^2), r0 = 180/pi
        phi = atan2(-u', v'), theta = atan2(r0, r)
        dec = asin(sin th sin dec0 + cos th cos dec0 cos phi)
        ra  = ra0 + atan2(-cos th sin phi, sin th cos dec0 - cos th sin dec0 cos phi)

    Sec. 3.2.2 (source WCS, world -> pixel)
        dra = ra - ra0
        phi   = atan2(-cos dec sin dra, sin dec cos dec0 - cos dec sin dec0 cos dra)
        theta = asin(sin dec sin dec0 + cos dec cos dec0 cos dra)
        r = r0 cos th / sin th, u' = -r sin phi, v' = r cos phi
        (u, v) = CD^-1 (u', v'); inverse SIP AP/BP; x = u + (crpix1 - 1), y = v + (crpix2 - 1)

Readings taken where the paper is ambiguous (each is listed in the design notes):
  * SIP sign and update order: the paper prints ``u = u - SIP_A(u, v)``; the SIP convention it
    cites (Shupe et al. 2005) adds the polynomial, u <- u + A(u, v), v <- v + B(u, v), with both
    evaluated at the undistorted (u, v). The same holds for AP/BP on the way back.
  * SIP terms are the monomials u^p v^q with 1 <= p+q <= ORDER (no constant term), so the
    reference pixel maps to the reference value exactly.
  * The two ``asin`` steps (dec in Sec. 3.2.1, theta in Sec. 3.2.2) lose accuracy where their
    argument nears 1: d(angle) = d(arg) / cos(angle), i.e. ~1e-6 px one pixel from CRPIX for
    theta and ~1e-8 px near a pole for dec. Each argument is the third component of a unit
    vector whose other two components are exactly the two atan2 arguments printed beside it
    (cos th sin phi, cos th cos phi for theta; the ra arguments for dec), so the oracle computes
    the same angle as atan2(z, hypot(x, y)). ``theta_mode="asin"`` keeps the printed form.
  * A target point is covered by the source only where the source sin(theta) > 0.
  * LONPOLE (the native longitude of the celestial pole, phi_p) is 180 deg in the paper's
    formulas. A record may carry another value as ``lonpole``: the rotation steps then use
    phi - (phi_p - 180 deg) in place of phi (the paper's phi is the standard native longitude
    minus 180 deg), as in the general zenithal case of FITS WCS Paper II.

All functions are written over a math namespace ``m`` (numpy by default) so that the same code
runs on forward-mode dual numbers (oracle.dual) for gradients.
"""
from __future__ import annotations

import math
import re

import numpy as np

R0 = 180.0 / math.pi
DEG = math.pi / 180.0
MAX_SIP = 9


# ------------------------------------------------------------------------------ SIP
def sip_value(coef, order, u, v):
    """Sum of coef[p][q] u^p v^q over 1 <= p+q <= order (Shupe et al. 2005, Eq. 1-2)."""
    total = 0.0 * u
    for p in range(order + 1):
        for q in range(order + 1 - p):
            if p + q == 0:
                continue
            c = coef[p][q]
            if isinstance(c, float) and c == 0.0:
                continue
            total = total + c * (u ** p) * (v ** q)
    return total


def sip_partials(coef, order, u, v):
    """(d/du, d/dv) of sip_value, differentiated term by term."""
    du = 0.0 * u
    dv = 0.0 * u
    for p in range(order + 1):
        for q in range(order + 1 - p):
            if p + q == 0:
                continue
            c = coef[p][q]
            if isinstance(c, float) and c == 0.0:
                continue
            if p > 0:
                du = du + c * p * (u ** (p - 1)) * (v ** q)
            if q > 0:
                dv = dv + c * q * (u ** p) * (v ** (q - 1))
    return du, dv


def _coef(w, name):
    c = w[name]
    if isinstance(c, np.ndarray):
        return [[float(c[p, q]) for q in range(c.shape[1])] for p in range(c.shape[0])]
    return c


# ------------------------------------------------------------------------------ CD
def cd_inverse(cd):
    """Inverse of the 2x2 CD matrix (Sec. 3.2.2), by the adjugate formula."""
    a, b = cd[0][0], cd[0][1]
    c, d = cd[1][0], cd[1][1]
    det = a * d - b * c
    return [[d / det, -b / det], [-c / det, a / det]]


def _lonpole_offset(w):
    """phi_p - 180 deg in radians (0 for the paper's phi_p = 180 deg)."""
    return (float(w.get("lonpole", 180.0)) - 180.0) * DEG


# ------------------------------------------------------------------------------ Sec. 3.2.1
def pix2world(w, x, y, m=np, theta_mode="atan2"):
    """Target pixel (0-based x, y) -> (ra, dec) in degrees, Sec. 3.2.1."""
    crpix1, crpix2 = w["crpix"]
    ra0 = w["crval"][0] * DEG
    dec0 = w["crval"][1] * DEG
    cd = w["cd"]
    # shift (0-based pixels)
    u = x - (crpix1 - 1.0)
    v = y - (crpix2 - 1.0)
    # SIP distortion, both polynomials at the undistorted (u, v)
    if w["a_order"] > 0 or w["b_order"] > 0:
        fu = sip_value(_coef(w, "a"), w["a_order"], u, v)
        fv = sip_value(_coef(w, "b"), w["b_order"], u, v)
        u, v = u + fu, v + fv
    # CD matrix -> intermediate world coordinates in degrees
    up = cd[0][0] * u + cd[0][1] * v
    vp = cd[1][0] * u + cd[1][1] * v
    # gnomonic deprojection to native spherical coordinates
    r = m.sqrt(up * up + vp * vp)
    phi = m.arctan2(-up, vp) - _lonpole_offset(w)
    theta = m.arctan2(R0 + 0.0 * r, r)
    # native -> celestial
    st, ct = m.sin(theta), m.cos(theta)
    sp, cp = m.sin(phi), m.cos(phi)
    z = st * math.sin(dec0) + ct * math.cos(dec0) * cp
    ya = -ct * sp
    xa = st * math.cos(dec0) - ct * math.sin(dec0) * cp
    if theta_mode == "asin":
        dec = m.arcsin(z)
    else:
        dec = m.arctan2(z, m.sqrt(ya * ya + xa * xa))
    ra = ra0 + m.arctan2(ya, xa)
    return ra / DEG, dec / DEG


# ------------------------------------------------------------------------------ Sec. 3.2.2
def world_to_intermediate(w, ra_deg, dec_deg, m=np, theta_mode="atan2"):
    """(ra, dec) -> source intermediate pixel offsets (u, v) = CD^-1 (u', v') before inverse SIP.

    Returns (u, v, valid) where valid marks sin(theta) > 0 (the point is on the source's
    projection hemisphere)."""
    ra0 = w["crval"][0] * DEG
    dec0 = w["crval"][1] * DEG
    ra = ra_deg * DEG
    dec = dec_deg * DEG
    dra = ra - ra0
    sd, cdn = m.sin(dec), m.cos(dec)
    sdra, cdra = m.sin(dra), m.cos(dra)
    sd0, cd0 = m.sin(dec0), m.cos(dec0)
    n1 = -cdn * sdra
    n2 = sd * cd0 - cdn * sd0 * cdra
    dd = sd * sd0 + cdn * cd0 * cdra
    phi = m.arctan2(n1, n2) + _lonpole_offset(w)
    if theta_mode == "asin":
        theta = m.arcsin(dd)
    else:
        theta = m.arctan2(dd, m.sqrt(n1 * n1 + n2 * n2))
    st = m.sin(theta)
    r = R0 * m.cos(theta) / st
    up = -r * m.sin(phi)
    vp = r * m.cos(phi)
    ci = cd_inverse(w["cd"])
    u = ci[0][0] * up + ci[0][1] * vp
    v = ci[1][0] * up + ci[1][1] * vp
    valid = np.asarray(_val(st)) > 0.0
    return u, v, valid


def _val(a):
    return a.v if hasattr(a, "v") and hasattr(a, "d") else a


def inverse_sip_poly(w, u, v):
    """Apply AP/BP to (u, v): u + AP(u, v), v + BP(u, v) (both at the input point)."""
    if w["ap_order"] <= 0 and w["bp_order"] <= 0:
        return u, v
    gu = sip_value(_coef(w, "ap"), w["ap_order"], u, v)
    gv = sip_value(_coef(w, "bp"), w["bp_order"], u, v)
    return u + gu, v + gv


def inverse_sip_newton(w, U, V, tol=1e-12, max_iter=30, extra=2):
    """Exact inverse of the forward SIP: solve u + A(u, v) = U, v + B(u, v) = V by Newton's
    method, starting from the AP/BP polynomial when present. Stops once every step is below
    ``tol`` px, then takes ``extra`` more steps (so dual-number derivatives converge too)."""
    if w["a_order"] <= 0 and w["b_order"] <= 0:
        return U, V
    a, b = _coef(w, "a"), _coef(w, "b")
    u, v = inverse_sip_poly(w, U, V)
    left = None
    for _ in range(max_iter):
        fu = u + sip_value(a, w["a_order"], u, v) - U
        fv = v + sip_value(b, w["b_order"], u, v) - V
        au, av = sip_partials(a, w["a_order"], u, v)
        bu, bv = sip_partials(b, w["b_order"], u, v)
        j00, j01 = 1.0 + au, av
        j10, j11 = bu, 1.0 + bv
        det = j00 * j11 - j01 * j10
        du = (j11 * fu - j01 * fv) / det
        dv = (j00 * fv - j10 * fu) / det
        u = u - du
        v = v - dv
        step = np.nanmax(np.abs(np.concatenate([np.ravel(_val(du)), np.ravel(_val(dv))])))
        if left is None and step < tol:
            left = extra
        if left is not None:
            if left == 0:
                break
            left -= 1
    return u, v


def world2pix(w, ra_deg, dec_deg, inverse="poly", m=np, theta_mode="atan2"):
    """(ra, dec) in degrees -> source pixel (0-based x, y), Sec. 3.2.2.

    inverse="poly" applies AP/BP; inverse="newton" solves the forward A/B exactly.
    Returns (x, y, valid)."""
    u, v, valid = world_to_intermediate(w, ra_deg, dec_deg, m=m, theta_mode=theta_mode)
    if inverse == "newton":
        u, v = inverse_sip_newton(w, u, v)
    else:
        u, v = inverse_sip_poly(w, u, v)
    crpix1, crpix2 = w["crpix"]
    x = u + (crpix1 - 1.0)
    y = v + (crpix2 - 1.0)
    return x, y, valid


def source_coords(src, tgt, x_t, y_t, inverse="poly", m=np, theta_mode="atan2"):
    """Target pixel -> source pixel: Sec. 3.1 steps 1 and 2."""
    ra, dec = pix2world(tgt, x_t, y_t, theta_mode=theta_mode)
    return world2pix(src, ra, dec, inverse=inverse, m=m, theta_mode=theta_mode)


# ------------------------------------------------------------------------------ AP/BP fit
def fit_inverse_sip(w, order, ngrid=100, margin=0.05, check_grid=512):
    """Least-squares inverse SIP of the given order (monomials 1 <= p+q <= order).

    Samples a ngrid x ngrid grid over the frame plus a fractional margin, maps it through the
    forward SIP, and fits u - U = AP(U, V), v - V = BP(U, V) with Householder QR on
    coordinates scaled by R = half the larger side. Returns (ap, bp, stats) where stats holds
    the max and RMS round-trip residual (px) over a check_grid^2 grid of the frame."""
    W, H = w["naxis"]
    a, b = _coef(w, "a"), _coef(w, "b")
    R = max(W, H) / 2.0
    xs = np.linspace(-margin * W - 0.5, (1.0 + margin) * W - 0.5, ngrid)
    ys = np.linspace(-margin * H - 0.5, (1.0 + margin) * H - 0.5, ngrid)
    X, Y = np.meshgrid(xs, ys)
    u = X.ravel() - (w["crpix"][0] - 1.0)
    v = Y.ravel() - (w["crpix"][1] - 1.0)
    U = u + sip_value(a, w["a_order"], u, v)
    V = v + sip_value(b, w["b_order"], u, v)
    terms = [(p, n - p) for n in range(1, order + 1) for p in range(n, -1, -1)]
    M = np.stack([(U / R) ** p * (V / R) ** q for (p, q) in terms], axis=1)
    Q, Rm = np.linalg.qr(M)
    import scipy.linalg
    cu = scipy.linalg.solve_triangular(Rm, Q.T @ (u - U))
    cv = scipy.linalg.solve_triangular(Rm, Q.T @ (v - V))
    ap = np.zeros((MAX_SIP + 1, MAX_SIP + 1))
    bp = np.zeros((MAX_SIP + 1, MAX_SIP + 1))
    for k, (p, q) in enumerate(terms):
        ap[p, q] = cu[k] / R ** (p + q)
        bp[p, q] = cv[k] / R ** (p + q)
    # round-trip residual on a check grid of the frame itself
    xs = np.linspace(-0.5, W - 0.5, check_grid)
    ys = np.linspace(-0.5, H - 0.5, check_grid)
    X, Y = np.meshgrid(xs, ys)
    u = X.ravel() - (w["crpix"][0] - 1.0)
    v = Y.ravel() - (w["crpix"][1] - 1.0)
    U = u + sip_value(a, w["a_order"], u, v)
    V = v + sip_value(b, w["b_order"], u, v)
    ap_l = [[float(ap[i, j]) for j in range(MAX_SIP + 1)] for i in range(MAX_SIP + 1)]
    bp_l = [[float(bp[i, j]) for j in range(MAX_SIP + 1)] for i in range(MAX_SIP + 1)]
    ru = U + sip_value(ap_l, order, U, V) - u
    rv = V + sip_value(bp_l, order, U, V) - v
    res = np.hypot(ru, rv)
    return ap, bp, {"max_px": float(res.max()), "rms_px": float(np.sqrt(np.mean(res ** 2)))}


def with_inverse_sip(w, order, **kw):
    """Copy of the WCS record with AP/BP fitted by fit_inverse_sip."""
    out = dict(w)
    ap, bp, stats = fit_inverse_sip(w, order, **kw)
    out["ap"], out["bp"] = ap, bp
    out["ap_order"] = out["bp_order"] = order
    out["cd"] = [list(w["cd"][0]), list(w["cd"][1])]
    out["a"], out["b"] = np.array(w["a"]), np.array(w["b"])
    return out, stats


# ------------------------------------------------------------------------------ header
class HeaderError(ValueError):
    pass


def _records(text):
    if "\n" in text:
        return [ln.rstrip("\r") for ln in text.split("\n")]
    return [text[i:i + 80] for i in range(0, len(text), 80)]


def _parse_value(s):
    s = s.strip()
    if s.startswith("'"):
        end = s.find("'", 1)
        while end != -1 and end + 1 < len(s) and s[end + 1] == "'":
            end = s.find("'", end + 2)
        if end == -1:
            raise HeaderError("unterminated string")
        return s[1:end].replace("''", "'").rstrip()
    slash = s.find("/")
    if slash >= 0:
        s = s[:slash].strip()
    if s in ("T", "F"):
        return s == "T"
    if re.fullmatch(r"[+-]?\d+", s):
        return int(s)
    try:
        return float(s.replace("D", "E").replace("d", "e"))
    except ValueError as exc:
        raise HeaderError("bad value %r" % s) from exc


def parse_header(text):
    """FITS header cards -> WCS record. CD wins over PC x CDELT, which wins over CDELT with the
    legacy CROTA2 rotation; LONPOLE other than 180 is kept in the record (``lonpole``); CTYPE
    must be RA---TAN / DEC--TAN with an optional -SIP suffix."""
    cards = {}
    for rec in _records(text):
        key = rec[:8].strip()
        if not key or key in ("END", "COMMENT", "HISTORY"):
            continue
        if rec[8:10] != "= ":
            continue
        cards[key] = _parse_value(rec[10:])
    for k in ("NAXIS1", "NAXIS2", "CRPIX1", "CRPIX2", "CRVAL1", "CRVAL2", "CTYPE1", "CTYPE2"):
        if k not in cards:
            raise HeaderError("missing " + k)
    c1, c2 = str(cards["CTYPE1"]), str(cards["CTYPE2"])
    if c1[:8] != "RA---TAN" or c2[:8] != "DEC--TAN" or c1[8:] not in ("", "-SIP") \
            or c2[8:] not in ("", "-SIP"):
        raise HeaderError("unsupported CTYPE")
    for k in ("LONPOLE", "CROTA2"):
        if k in cards and (isinstance(cards[k], (str, bool))):
            raise HeaderError("%s is not a number" % k)
    lonpole = float(cards.get("LONPOLE", 180.0))
    if not math.isfinite(lonpole):
        raise HeaderError("bad LONPOLE")
    has_pc = any(k in cards for k in ("PC1_1", "PC1_2", "PC2_1", "PC2_2"))
    if any(k in cards for k in ("CD1_1", "CD1_2", "CD2_1", "CD2_2")):
        cd = [[float(cards.get("CD1_1", 0.0)), float(cards.get("CD1_2", 0.0))],
              [float(cards.get("CD2_1", 0.0)), float(cards.get("CD2_2", 0.0))]]
    elif "CDELT1" in cards and "CDELT2" in cards:
        d = [float(cards["CDELT1"]), float(cards["CDELT2"])]
        if not has_pc and "CROTA2" in cards:
            # legacy AIPS rotation (FITS WCS Paper II, Sec. 6.1): CD = diag(CDELT) rotated
            rho = float(cards["CROTA2"]) * DEG
            cd = [[d[0] * math.cos(rho), -d[1] * math.sin(rho)],
                  [d[0] * math.sin(rho), d[1] * math.cos(rho)]]
        else:
            pc = [[float(cards.get("PC1_1", 1.0)), float(cards.get("PC1_2", 0.0))],
                  [float(cards.get("PC2_1", 0.0)), float(cards.get("PC2_2", 1.0))]]
            cd = [[d[0] * pc[0][0], d[0] * pc[0][1]], [d[1] * pc[1][0], d[1] * pc[1][1]]]
    else:
        raise HeaderError("no CD or CDELT")
    if cd[0][0] * cd[1][1] - cd[0][1] * cd[1][0] == 0.0:
        raise HeaderError("singular CD")
    w = {
        "naxis": (int(cards["NAXIS1"]), int(cards["NAXIS2"])),
        "crpix": (float(cards["CRPIX1"]), float(cards["CRPIX2"])),
        "crval": (float(cards["CRVAL1"]), float(cards["CRVAL2"])),
        "cd": cd,
    }
    if lonpole != 180.0:
        w["lonpole"] = lonpole
    for name in ("A", "B", "AP", "BP"):
        order = int(cards.get(name + "_ORDER", 0))
        if order < 0 or order > MAX_SIP:
            raise HeaderError("bad %s_ORDER" % name)
        coef = np.zeros((MAX_SIP + 1, MAX_SIP + 1))
        for p in range(order + 1):
            for q in range(order + 1 - p):
                key = "%s_%d_%d" % (name, p, q)
                if key in cards and p + q >= 1:
                    coef[p, q] = float(cards[key])
        w[name.lower() + "_order"] = order
        w[name.lower()] = coef
    return w
