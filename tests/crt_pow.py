"""x^e mod N through the CRT over N's known prime factors, with CPython's pow (a check independent
of the library and of the oracle's own square-and-multiply).  A module of its own so that a spawned
process pool can import it."""


def crt_modexp(args):
    x, e, p, q = args
    N = p * q
    if e == 0:
        return 1 % N
    rp = 0 if x % p == 0 else pow(x, e % (p - 1), p)
    rq = 0 if x % q == 0 else pow(x, e % (q - 1), q)
    h = (rp - rq) * pow(q, -1, p) % p
    return rq + h * q
